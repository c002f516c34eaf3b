"""Write median_sel.cuh: branch-free median-selection networks for 9, 25 and
49 values, each derived here from Batcher's odd-even merge sort.

1. Batcher's network for P = the next power of two >= N.
2. Inputs N .. P-1 would be +inf padding.  A padded wire always holds +inf
   (a comparator puts the larger value on its higher wire), so every
   comparator that touches one is a no-op and is dropped.
3. Only the middle output, wire (N - 1) / 2, is wanted.  Walking the
   comparators backwards with the set of wires still needed, a comparator
   with neither output needed is dropped, one with only its lower output
   needed becomes v_i = min(v_i, v_j), one with only its upper output needed
   becomes v_j = max(v_i, v_j), and one with both stays a compare-exchange.

The result selects the same order statistic as sorting the N values, for
inputs without NaN.  Run: python gen_median.py  (writes median_sel.cuh
beside this file).
"""
import os


def batcher(p):
    """Comparators (i, j), i < j, of Batcher's odd-even merge sort of p = 2^k wires, in order."""
    out = []

    def merge(lo, n, r):
        step = r * 2
        if step < n:
            merge(lo, n, step)
            merge(lo + r, n, step)
            i = lo + r
            while i + r < lo + n:
                out.append((i, i + r))
                i += step
        else:
            out.append((lo, lo + r))

    def sort(lo, n):
        if n > 1:
            sort(lo, n // 2)
            sort(lo + n // 2, n // 2)
            merge(lo, n, 1)

    sort(0, p)
    return out


def selection(n):
    p = 1
    while p < n:
        p *= 2
    net = [(i, j) for i, j in batcher(p) if j < n]
    need = {(n - 1) // 2}
    ops = []
    for i, j in reversed(net):
        ni, nj = i in need, j in need
        if ni and nj:
            ops.append(("x", i, j))
        elif ni:
            ops.append(("min", i, j))
            need.add(j)
        elif nj:
            ops.append(("max", i, j))
            need.add(i)
    ops.reverse()
    return ops


def check(n, ops, trials=20000):
    import random
    rng = random.Random(n)
    for _ in range(trials):
        v = [rng.choice([rng.random(), rng.randint(0, 5)]) for _ in range(n)]
        w = list(v)
        for kind, i, j in ops:
            a, b = w[i], w[j]
            if kind == "x":
                w[i], w[j] = min(a, b), max(a, b)
            elif kind == "min":
                w[i] = min(a, b)
            else:
                w[j] = max(a, b)
        assert w[(n - 1) // 2] == sorted(v)[(n - 1) // 2]


def render():
    """The text of median_sel.cuh."""
    lines = ["// median_sel.cuh -- written by gen_median.py (do not edit): median-selection",
             "// networks pruned from Batcher's odd-even merge sort (see gen_median.py).",
             "// med_sel<N>(v) returns the middle value of v[0 .. N-1] (N odd, no NaN);",
             "// v is overwritten.",
             "#pragma once", "", "namespace gp {", "",
             "template <int N>", "__device__ __forceinline__ float med_sel(float (&v)[N]);", ""]
    for n in (9, 25, 49):
        ops = selection(n)
        check(n, ops)
        nx = sum(1 for o in ops if o[0] == "x")
        lines += [f"// {n} values: {len(ops)} comparators, {nx} of them full compare-exchanges",
                  "template <>", f"__device__ __forceinline__ float med_sel<{n}>(float (&v)[{n}])", "{"]
        for kind, i, j in ops:
            if kind == "x":
                lines.append(f"    {{ const float a = v[{i}], b = v[{j}]; v[{i}] = fminf(a, b); v[{j}] = fmaxf(a, b); }}")
            elif kind == "min":
                lines.append(f"    v[{i}] = fminf(v[{i}], v[{j}]);")
            else:
                lines.append(f"    v[{j}] = fmaxf(v[{i}], v[{j}]);")
        lines += [f"    return v[{(n - 1) // 2}];", "}", ""]
    lines += ["}  // namespace gp", ""]
    return "\n".join(lines)


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    open(os.path.join(here, "median_sel.cuh"), "w").write(render())


if __name__ == "__main__":
    main()
