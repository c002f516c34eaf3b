"""The median-selection networks of the cosmetic filters (Section 3.1):
each, run on the host, selects the middle order statistic of its inputs,
and the committed header is the generator's output."""
import importlib.util
import os
import random

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2609_32375_gb300", "csrc")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_median", os.path.join(CSRC, "gen_median.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _run(ops, v):
    w = list(v)
    for kind, i, j in ops:
        a, b = w[i], w[j]
        if kind == "x":
            w[i], w[j] = min(a, b), max(a, b)
        elif kind == "min":
            w[i] = min(a, b)
        else:
            w[j] = max(a, b)
    return w


@pytest.mark.parametrize("n", [9, 25, 49])
def test_network_selects_the_median(n):
    """Random values, many ties, sorted and reversed inputs, and every 0/1
    input with a few ones or zeros (a selection network is correct on all
    inputs when it is on all 0/1 inputs; this samples them)."""
    g = _gen()
    ops = g.selection(n)
    m = (n - 1) // 2
    rng = random.Random(n)
    cases = [sorted(range(n)), sorted(range(n), reverse=True)]
    cases += [[rng.random() for _ in range(n)] for _ in range(3000)]
    cases += [[rng.randint(0, 3) for _ in range(n)] for _ in range(3000)]
    for k in range(n + 1):
        for _ in range(40):
            v = [1] * k + [0] * (n - k)
            rng.shuffle(v)
            cases.append(v)
    for v in cases:
        assert _run(ops, v)[m] == sorted(v)[m]


def test_network_sizes():
    """Fewer comparisons than Batcher's full sort of the padded inputs."""
    g = _gen()
    for n, p in ((9, 16), (25, 32), (49, 64)):
        full = len(g.batcher(p))
        assert len(g.selection(n)) < full


def test_header_is_the_generator_output():
    g = _gen()
    assert open(os.path.join(CSRC, "median_sel.cuh")).read() == g.render()
