"""Host-side checks of the batched regression workload recipe (no GPU)."""
import collections
import math

import workloads as W


def test_batch_shapes_follow_the_recipe():
    sh = W.batch_shapes(512, seed=7)
    assert len(sh) == 512
    assert [s["seed"] for s in sh] == list(range(1, 513))
    assert all(2 ** 12 <= s["n"] < 2 ** 18 for s in sh)
    assert all(s["m"] == 4 * s["d"] ** 2 for s in sh)
    assert all(s["kmin"] == 4 and s["kmax"] == min(32, s["d"]) for s in sh)
    cnt = collections.Counter(s["d"] for s in sh)
    assert set(cnt) == {16, 32, 64, 128} and min(cnt.values()) > 90
    # log-uniform n: about half the problems below 2^15
    below = sum(1 for s in sh if s["n"] < 2 ** 15)
    assert 200 < below < 312
    assert W.batch_shapes(512, seed=7) == sh


def test_batch_problem_rows():
    s = dict(n=3000, d=16, m=1024, kmin=4, kmax=16, seed=3)
    A, b = W.batch_problem(s)
    lens = (A.row_ptr[1:] - A.row_ptr[:-1]).numpy()
    assert A.n == 3000 and b.shape == (3000,)
    assert lens.min() >= 4 and lens.max() <= 16
    rp, c, _ = A.numpy()
    for i in range(0, 3000, 97):
        row = c[rp[i]:rp[i + 1]]
        assert len(set(row.tolist())) == len(row) and (row >= 0).all() and (row < 16).all()
    A2, b2 = W.batch_problem(s)
    assert (A2.col == A.col).all() and (b2 == b).all()
    assert not math.isnan(float(b.sum()))
