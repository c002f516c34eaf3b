"""Checkpoint and resume of the learned background's training loop (no GPU).

The training state -- master weights, biases, AdamW moments, step count,
finished epochs and their losses -- goes to one file after every epoch, and
a run that finds the file continues after its last finished epoch.  The
GPU network is stood in for by a CPU model with the same state layout and a
deterministic update whose result depends on every piece of that state and
on the order of the minibatches, so a resume that lost any of it, or drew
other permutations, would end with different weights."""
import math

import pytest

torch = pytest.importorskip("torch")
from paper_2609_32375_gb300 import learned  # noqa: E402


class CpuNet:
    """Same state lists as learned.Network; AdamW on a per-layer linear map."""

    def __init__(self, seed=0):
        g = torch.Generator().manual_seed(seed)
        self.W = [torch.randn(3, 4, generator=g, dtype=torch.float64) for _ in range(6)]
        self.b = [torch.randn(3, generator=g, dtype=torch.float64) for _ in range(6)]
        self.mW = [torch.zeros_like(w) for w in self.W]
        self.vW = [torch.zeros_like(w) for w in self.W]
        self.mb = [torch.zeros_like(b) for b in self.b]
        self.vb = [torch.zeros_like(b) for b in self.b]
        self.step = 0
        self.packs = 0

    def pack(self, stream=None):
        self.packs += 1

    def load_state_dict(self, d):
        learned.Network.load_state_dict(self, d)

    def train_step(self, feat, target, lr=2e-3, stream=None):
        self.step += 1
        b1, b2, eps = 0.9, 0.999, 1e-8
        loss = 0.0
        for l in range(6):
            pred = feat @ self.W[l].T + self.b[l]
            err = pred - target
            loss += float((err ** 2).mean())
            gW = 2 * err.T @ feat / err.numel()
            gb = 2 * err.mean(0)
            for p, gr, m, v in ((self.W[l], gW, self.mW[l], self.vW[l]), (self.b[l], gb, self.mb[l], self.vb[l])):
                m.mul_(b1).add_(gr, alpha=1 - b1)
                v.mul_(b2).addcmul_(gr, gr, value=1 - b2)
                mh = m / (1 - b1 ** self.step)
                vh = v / (1 - b2 ** self.step)
                p.sub_(lr * mh / (vh.sqrt() + eps))
        return torch.tensor(loss)


def _data(n=24):
    g = torch.Generator().manual_seed(7)
    feat = torch.randn(n, 4, generator=g, dtype=torch.float64)
    target = torch.randn(n, 3, generator=g, dtype=torch.float64)
    return {"feat": feat, "target": target}


def _same(a, b):
    for k in ("W", "b", "mW", "vW", "mb", "vb"):
        for x, y in zip(getattr(a, k), getattr(b, k)):
            assert torch.equal(x, y), k
    assert a.step == b.step


def test_resume_continues_exactly_as_the_uninterrupted_run(tmp_path):
    data = _data()
    ref = CpuNet()
    hist_ref = learned.train(ref, data, epochs=6, batch=4, lr=1e-2, seed=3)

    ck = str(tmp_path / "state.npz")
    first = CpuNet()
    hist_a = learned.train(first, data, epochs=6, batch=4, lr=1e-2, seed=3, checkpoint=ck)
    assert hist_a == hist_ref
    _same(first, ref)

    # interrupted after two epochs: a fresh process (a new network) resumes from the file
    ck2 = str(tmp_path / "part.npz")
    part = CpuNet()
    full_sched = dict(epochs=6, batch=4, lr=1e-2, seed=3)
    # run two epochs of the six-epoch schedule, then stop (as if killed)
    rec = {"epochs": 6, "batch": 4, "seed": 3, "n": data["feat"].shape[0], "losses": []}
    g = torch.Generator(device="cpu").manual_seed(3)
    for ep in range(2):
        perm = torch.randperm(rec["n"], generator=g)
        lr_e = 1e-2 * 0.5 * (1 + math.cos(math.pi * ep / 6))
        losses = [part.train_step(data["feat"][perm[s:s + 4]], data["target"][perm[s:s + 4]], lr=lr_e)
                  for s in range(0, rec["n"] - 4 + 1, 4)]
        rec["losses"].append(float(torch.stack(losses).mean()))
    learned.save_checkpoint(part, ck2, rec)
    assert rec["losses"] == hist_ref[:2]

    resumed = CpuNet(seed=99)                 # other initial weights: all of them must come from the file
    hist_b = learned.train(resumed, data, checkpoint=ck2, **full_sched)
    assert hist_b == hist_ref
    _same(resumed, ref)


def test_checkpoint_round_trip_and_schedule_guard(tmp_path):
    net = CpuNet()
    learned.train(net, _data(), epochs=2, batch=4, lr=1e-2, seed=1)
    ck = str(tmp_path / "s.npz")
    learned.save_checkpoint(net, ck, {"epochs": 2, "batch": 4, "seed": 1, "n": 24, "losses": [1.0, 0.5]})
    other = CpuNet(seed=5)
    rec = learned.load_checkpoint(other, ck)
    assert rec["losses"] == [1.0, 0.5]
    assert other.packs >= 1                   # packed forms rebuilt from the restored master weights
    _same(other, net)
    with pytest.raises(ValueError):
        learned.train(CpuNet(), _data(), epochs=3, batch=4, lr=1e-2, seed=1, checkpoint=ck)


def test_weights_only_files_leave_the_moments_at_zero():
    net = CpuNet()
    learned.train(net, _data(), epochs=1, batch=4, lr=1e-2, seed=0)
    fresh = CpuNet(seed=4)
    fresh.load_state_dict({"W": net.W, "b": net.b})
    assert all(torch.count_nonzero(m) == 0 for m in fresh.mW + fresh.vW + fresh.mb + fresh.vb)
    assert all(torch.equal(x, y) for x, y in zip(fresh.W, net.W))
