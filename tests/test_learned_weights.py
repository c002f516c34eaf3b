"""The committed weights of the learned background: each records the training
run it came from, and the lookup by mesh size finds the one trained at that
mesh (no GPU needed)."""
import numpy as np

from paper_2609_32375_gb300 import learned


def test_weights_carry_their_training_record():
    for mesh in (64, 256):
        path = learned.weights_for_mesh(mesh)
        assert path is not None, mesh
        m = learned.meta(path)
        assert m["mesh"] == mesh
        assert m["loss_last_epoch"] < 0.1 * m["loss_first_epoch"]
        z = np.load(path)
        # six 3x3 layers, 5 feature channels in (padded) and 2 out
        assert sum(1 for k in z.files if k.startswith("W")) == 6
        assert all(np.all(np.isfinite(z[k])) for k in z.files if k != "meta")


def test_no_weights_for_an_untrained_mesh():
    assert learned.weights_for_mesh(128) is None


def test_mesh256_weights_were_trained_on_uint16_frames_at_the_dense_density():
    m = learned.meta(learned.weights_for_mesh(256))
    assert m["u16"] is True
    # stars per frame of 8192^2 px: 30 .. 1,500 per megapixel (the dense recipe has 890)
    lo, hi = m["stars"]
    px = m["size"] ** 2 / 1e6
    assert lo / px <= 890 <= hi / px
