"""Device arithmetic against IEEE binary64 on the host, and the device's
exact orientation sign against the oracle's and rational arithmetic.

The quality functional (Sec. 2.2) takes means of three terms: the oracle
divides by 3.0; the library forms the same quotient by Markstein's
correction (one multiplication, two fused multiply-adds).  The two must agree
bit for bit on every double, so the check covers a large sample of random bit
patterns (every exponent, both signs, NaN and infinities included), values of
moderate size where the quality's inputs live, and the hard cases: zeros of
both signs, subnormals, powers of two and their neighbours, and values next
to the overflow threshold.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pm = pytest.importorskip("paper_1505_04694_gb300.pm")


def _edge_cases():
    v = [0.0, -0.0, np.inf, -np.inf, 5e-324, -5e-324, 1e-310, -1e-310,
         2.2250738585072014e-308, np.finfo(np.float64).max, -np.finfo(np.float64).max,
         1.0, 3.0, 6.0, 0.1, 1.0 / 3.0, 1e300, 1.5e-323]
    p2 = np.ldexp(1.0, np.arange(-1074, 1024))
    up, down = p2.copy(), p2.copy()
    v += list(p2)
    for _ in range(3):  # three neighbours on each side of every power of two
        up = np.nextafter(up, np.inf)
        down = np.nextafter(down, 0.0)
        v += list(up) + list(down)
    big = np.finfo(np.float64).max
    x = big
    for _ in range(64):
        x = np.nextafter(x, 0.0)
        v.append(x)
    a = np.array(v, dtype=np.float64)
    return np.concatenate([a, -a])


def test_division_by_three_is_the_ieee_quotient():
    rng = np.random.default_rng(20261203)
    raw = rng.integers(0, 2 ** 64, size=8_000_000, dtype=np.uint64).view(np.float64)
    moderate = rng.uniform(-1e7, 1e7, size=4_000_000) * np.exp2(
        rng.integers(-60, 60, size=4_000_000))
    x = np.concatenate([raw, moderate, _edge_cases()])
    dev = torch.device("cuda:0")
    xd = torch.from_numpy(x).to(dev)
    od = torch.empty_like(xd)
    pm.selftest_div3_dev(xd, od)
    torch.cuda.synchronize(dev)
    got = od.cpu().numpy()
    with np.errstate(invalid="ignore", over="ignore"):
        want = x / 3.0
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    bad = np.nonzero(got[~nan].view(np.uint64) != want[~nan].view(np.uint64))[0]
    assert bad.size == 0, (bad.size, x[~nan][bad[:5]])
    # multiplying by the double nearest 1/3 is NOT the quotient for about a
    # third of all doubles: the sample does tell the two apart
    approx = x[~nan] * (1.0 / 3.0)
    assert np.count_nonzero(approx.view(np.uint64) != want[~nan].view(np.uint64)) > 1_000_000


def test_orientation_sign_is_exact_on_the_device():
    """The device predicate behind every validity decision gives the sign of
    the exact determinant (rational arithmetic) and the oracle's sign, on
    nearly collinear triples (some far from the origin, where the rounded
    formula is often wrong), general and exactly collinear ones."""
    from oracle import oracle as O
    from tests.test_oracle_pins import _exact_orient, _orient_cases

    cases = _orient_cases(3000, 91)
    pts = np.array([[*p, *q, *r] for p, q, r in cases], dtype=np.float64)
    dev = torch.device("cuda:0")
    pd = torch.from_numpy(pts).to(dev)
    od = torch.empty(pts.shape[0], dtype=torch.int32, device=dev)
    pm.selftest_orient_dev(pd, od)
    torch.cuda.synchronize(dev)
    got = od.cpu().numpy()
    wrong = 0
    for i, (p, q, r) in enumerate(cases):
        e = _exact_orient(p, q, r)
        assert got[i] == e == O.orient_sign(p, q, r), (i, got[i], e)
        naive = float((q[0] - p[0]) * (r[1] - p[1]) - (q[1] - p[1]) * (r[0] - p[0]))
        wrong += int((naive > 0) - (naive < 0) != e)
    assert wrong > 50
