"""Index safety of the step kernels' region streams (D2Q9, D2Q16, D3Q27), checked on the CPU.

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


# D2Q16 step (region stream of k_q16_step): per axis the four departure offsets
# d_k = -(s c_k + u) dt with c_k = -+sqrt(3 -+ sqrt 6), their floors as reals, and the region
# taken only when max - min <= Q16_REGION_MAX - 4 and both floors lie within 2^20 (NaN fails
# every comparison); only then are the floors converted to int.
Q16_REGION_MAX = 6
Q16_THREADS = 128
C16 = [np.float32(c) for c in (-np.sqrt(3 + np.sqrt(6)), -np.sqrt(3 - np.sqrt(6)),
                               np.sqrt(3 - np.sqrt(6)), np.sqrt(3 + np.sqrt(6)))]


def cuda_fmin(a, b):
    """fmin / fmax of CUDA return the other operand when one is NaN."""
    if np.isnan(a):
        return b
    if np.isnan(b):
        return a
    return min(a, b)


def cuda_fmax(a, b):
    if np.isnan(a):
        return b
    if np.isnan(b):
        return a
    return max(a, b)


def to_int(x):
    """float -> int conversion as cvt.rzi.s32: truncation, saturation, NaN to 0."""
    if np.isnan(x):
        return 0
    return int(max(min(np.trunc(x), I32.max), I32.min))


def check_axis_q16(s, u, dt, X=7):
    with np.errstate(all="ignore"):
        fl = [np.floor(-(np.float32(s) * c + np.float32(u)) * np.float32(dt)) for c in C16]
        flo = cuda_fmin(cuda_fmin(fl[0], fl[1]), cuda_fmin(fl[2], fl[3]))
        fhi = cuda_fmax(cuda_fmax(fl[0], fl[1]), cuda_fmax(fl[2], fl[3]))
        taken = bool(fhi - flo <= np.float32(Q16_REGION_MAX - 4)) and bool(abs(flo) <= 2.0 ** 20) \
            and bool(abs(fhi) <= 2.0 ** 20)
    if not taken:
        return False
    lo = X + to_int(flo) - 1
    side = to_int(fhi - flo) + 4
    assert 4 <= side <= Q16_REGION_MAX
    assert I32.min < lo - 1 and lo + side < I32.max
    with np.errstate(all="ignore"):
        for f in fl:   # a NaN floor (not reachable from a real gauge) converts to 0
            o = to_int(f - flo)
            assert 0 <= o <= side - 4
    for axis in range(2):
        for k in range(4):
            for c in range(Q16_REGION_MAX):
                e = (axis * 4 + k) * Q16_REGION_MAX + c
                assert 0 <= e < 2 * 4 * Q16_REGION_MAX
                assert e * Q16_THREADS + Q16_THREADS - 1 < 2 * 4 * Q16_REGION_MAX * Q16_THREADS
    # the node's own entry, when skipped, is an index of the region
    cxo = X - lo
    if 0 <= cxo < side:
        assert 0 <= cxo * side + cxo < side * side
    return True


def test_d2q16_region_indices_stay_in_the_tables():
    rng = np.random.default_rng(12)
    specials = [0.0, 1e-30, 1e-7, 0.05, 0.5, 1.0, 3.0, 1e3, 1e10, 1e38, np.inf, -np.inf, np.nan]
    taken = 0
    for s in [abs(x) if not np.isnan(x) else x for x in specials]:
        for u in specials + [-x for x in specials[1:-1]]:
            for dt in (0.146, 0.5, 1.0):
                taken += check_axis_q16(s, u, dt)
    for _ in range(3000):
        s = float(np.exp(rng.uniform(-10, 2)))
        u = float(rng.normal(0.0, 1.0))
        taken += check_axis_q16(s, u, float(rng.uniform(0.01, 1.0)))
    assert taken > 1000


# D3Q27 step (region stream of k_q27_step): per axis the three departure offsets
# d_k = -(s (k - 1) + u) dt, the same real-valued checks as D2Q16 with Q27_REGION_MAX = 6;
# the x table is zero-padded (3 x 6 entries), the y and z tables hold the four cubic
# weights per component (3 x 4 entries each) and are read only at j = c - offset in [0, 4).
Q27_REGION_MAX = 6
Q27_ENTRIES = 3 * Q27_REGION_MAX + 2 * 12


def check_axis_q27(s, u, dt, X=5):
    with np.errstate(all="ignore"):
        fl = [np.floor(-(np.float32(s) * np.float32(k - 1) + np.float32(u)) * np.float32(dt)) for k in range(3)]
        flo = cuda_fmin(cuda_fmin(fl[0], fl[1]), fl[2])
        fhi = cuda_fmax(cuda_fmax(fl[0], fl[1]), fl[2])
        taken = bool(fhi - flo <= np.float32(Q27_REGION_MAX - 4)) and bool(abs(flo) <= 2.0 ** 20) \
            and bool(abs(fhi) <= 2.0 ** 20)
    if not taken:
        return False
    lo = X + to_int(flo) - 1
    side = to_int(fhi - flo) + 4
    assert 4 <= side <= Q27_REGION_MAX
    assert I32.min < lo - 1 and lo + side < I32.max
    with np.errstate(all="ignore"):
        offs = [to_int(f - flo) for f in fl]
    for o in offs:
        assert 0 <= o <= side - 4
    for k in range(3):
        for c in range(Q27_REGION_MAX):            # padded x entries
            assert 0 <= k * Q27_REGION_MAX + c < 3 * Q27_REGION_MAX
        for c in range(side):                      # unpadded y / z entries, read only in range
            j = c - offs[k]
            if 0 <= j < 4:
                for axis in (1, 2):
                    e = 3 * Q27_REGION_MAX + (axis - 1) * 12 + k * 4 + j
                    assert 3 * Q27_REGION_MAX <= e < Q27_ENTRIES
    return True


def test_d3q27_region_indices_stay_in_the_tables():
    rng = np.random.default_rng(13)
    specials = [0.0, 1e-30, 1e-7, 0.05, 0.5, 1.0, 3.0, 1e3, 1e10, 1e38, np.inf, -np.inf, np.nan]
    taken = 0
    for s in [abs(x) if not np.isnan(x) else x for x in specials]:
        for u in specials + [-x for x in specials[1:-1]]:
            for dt in (0.228, 0.5, 1.0):
                taken += check_axis_q27(s, u, dt)
    for _ in range(3000):
        s = float(np.exp(rng.uniform(-10, 1)))
        u = float(rng.normal(0.0, 1.0))
        taken += check_axis_q27(s, u, float(rng.uniform(0.01, 1.0)))
    assert taken > 1000
    # the own-entry index of a region of sides W, H, D stays below W H D
    for W in range(4, Q27_REGION_MAX + 1):
        for H in range(4, Q27_REGION_MAX + 1):
            for D in range(4, Q27_REGION_MAX + 1):
                assert ((D - 1) * H + (H - 1)) * W + (W - 1) < W * H * D
