"""Index safety of the step kernel's region stream, checked on the CPU.

The kernel computes, per node and axis, the departure offsets d_j = -(s c_j + u) dt of the
three directions (clamped to +-2^20 nodes, NaN to the lower bound), their floors, the
region side 4 + max - min, and for region entry r the column/row (r + 0.5) / side.  This
test restates that index arithmetic in float32/int32 and checks, for adversarial gauges
(NaN, +-Inf, huge and tiny values, random ones), that whenever the region path is taken
every table index lies in [0, REGION_MAX) and every stencil position maps into the
region, and that the fallback's offsets stay in int32 range."""
import numpy as np

REGION_MAX = 8
LIM = np.float32(1048576.0)
I32 = np.iinfo(np.int32)


def clamp_offset(d):
    d = np.float32(d)
    if np.isnan(d):
        return -LIM
    return np.float32(min(max(d, -LIM), LIM))


def region(s, u, dt):
    fl, xi = [], []
    for j in range(3):
        with np.errstate(all="ignore"):
            d = clamp_offset(-(np.float32(s) * np.float32(j - 1) + np.float32(u)) * np.float32(dt))
        f = np.floor(d)
        assert I32.min < f < I32.max
        fl.append(int(f))
        xi.append(np.float32(d - f + np.float32(1)))
    side = 4 + max(fl) - min(fl)
    return fl, xi, side


def check_axis(s, u, dt):
    fl, xi, side = region(s, u, dt)
    assert side >= 4
    if side > REGION_MAX:
        for f in fl:                        # fallback path: x0 = X + f - 1 stays in range
            assert abs(f) <= 1048576
        return
    lo = min(fl)
    for j in range(3):                      # each direction's 4-node stencil inside the region
        o = fl[j] - lo
        assert 0 <= o and o + 3 < side
    inc = np.float32(1.0) / np.float32(side)
    for other in range(4, REGION_MAX + 1):
        n = side * other
        for r in range(n):
            cy = int(np.float32(np.float32(r) + np.float32(0.5)) * inc)
            cx = r - cy * side
            assert 0 <= cx < side <= REGION_MAX and 0 <= cy < other


def test_region_indices_stay_in_the_tables():
    rng = np.random.default_rng(11)
    specials = [0.0, 1e-30, 1e-7, 0.05, 0.5, 1.0, 3.0, 1e3, 1e10, 1e38, np.inf, -np.inf, np.nan]
    for s in [abs(x) if not np.isnan(x) else x for x in specials]:
        for u in specials + [-x for x in specials[1:-1]]:
            for dt in (0.146, 0.5, 1.0):
                check_axis(s, u, dt)
    for _ in range(3000):
        s = float(np.exp(rng.uniform(-10, 5)))
        u = float(rng.normal(0.0, 3.0))
        check_axis(s, u, float(rng.uniform(0.01, 1.0)))
