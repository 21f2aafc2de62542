"""The scoring kernel forms each task's rotation rows A = fl32(fl64(R / r))
(Sec. III-A's R = Rz(gamma) Ry(beta) Rx(alpha), the FP64 products and sums of
rotation_rows) from FP32 operations on double-float copies of the FP64
cos / sin values (rotation_rows_df), falling back to FP64 where the FP32
result cannot decide the rounding.  Emulated here step by step with IEEE
FP32 arithmetic (FMA exact), it must give the FP64 definition's bits wherever
it does not fall back: on the rotations of the room, indoor and outdoor pose
grids, on random angles, and on angles chosen to make entries cancel, vanish
or sit on rounding boundaries; and it must fall back rarely."""
import math
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2310_10023_gb300 import synth

f32 = np.float32


def _bits(x):
    return int(np.array(x, dtype=np.float32).view(np.uint32))


def _from_bits(b):
    return f32(np.array(b & 0xFFFFFFFF, dtype=np.uint32).view(np.float32))


# ---- IEEE FP32 operations (round to nearest even) ---------------------------
# Sums, differences and products of two floats rounded once from the FP64
# value are correctly rounded (53 >= 2 * 24 + 2); fma needs the exact sum.
def fadd(a, b):
    return f32(float(a) + float(b))


def fsub(a, b):
    return f32(float(a) - float(b))


def fmul(a, b):
    return f32(float(a) * float(b))


def _two_sum64(x, y):
    s = x + y
    bb = s - x
    return s, (x - (s - bb)) + (y - bb)


def fma(a, b, c):
    """fl32(a b + c): a b is exact in FP64; the FP64 sum s with its exact
    error e then decides the FP32 rounding (e only matters when s is an FP32
    rounding midpoint)."""
    s, e = _two_sum64(float(a) * float(b), float(c))
    r = f32(s)
    if math.isinf(r) or float(r) == s:
        return r if float(r) != 0.0 or e == 0.0 else f32(e)
    nb = np.nextafter(r, f32(math.copysign(math.inf, s - float(r))))
    mid = (float(r) + float(nb)) / 2.0          # exact in FP64
    if s != mid or e == 0.0:
        return r
    return r if (e > 0) == (float(r) > float(nb)) else nb


# ---- the double-float steps of rotation_rows_df -----------------------------
def df_split(x):
    """(h, l, in_range): h the leading 24 significand bits of x, l the other 29
    rounded to a float."""
    u = struct.unpack("<Q", struct.pack("<d", x))[0]
    hi, lo = u >> 32, u & 0xFFFFFFFF
    sgn = hi & 0x80000000
    if ((hi & 0x7FFFFFFF) | lo) == 0:
        return _from_bits(sgn), f32(0.0), True
    e = ((hi >> 20) & 0x7FF) - 1023
    ok = -60 <= e < 30
    ec = min(max(e, -60), 29)
    h = _from_bits(sgn | ((ec + 127) << 23) | ((hi & 0xFFFFF) << 3) | (lo >> 29))
    l = fmul(f32(lo & 0x1FFFFFFF), _from_bits((ec - 52 + 127) << 23))
    return h, (-l if sgn else l), ok


def df_mul(a, b):
    p = fmul(a[0], b[0])
    e = fma(a[0], b[0], -p)
    e = fma(a[0], b[1], e)
    e = fma(a[1], b[0], e)
    return p, e


def two_sum(a, b):
    s = fadd(a, b)
    bb = fsub(s, a)
    return s, fadd(fsub(a, fsub(s, bb)), fsub(b, bb))


def df_add(a, b):
    s = two_sum(a[0], b[0])
    return two_sum(s[0], fadd(fadd(s[1], a[1]), b[1]))


def df_round(v, D):
    hb = _bits(v[0])
    eb = hb & 0x7F800000
    ok = (40 << 23) <= eb < (215 << 23)
    half = _from_bits(max(eb, 40 << 23) - (24 << 23))
    if hb & 0x7FFFFF == 0:
        half = fmul(half, f32(0.5))
    return v[0], ok and fadd(abs(v[1]), D) < half


TOL = f32(2.0 ** -40)
TINY = f32(2.0 ** -100)


def rows_df(ca, sa, cb, sb, cg, sg, inv_r):
    """The emulated rotation_rows_df: (A, ok)."""
    ok = True
    sp = []
    for x in (ca, sa, cb, sb, cg, sg, inv_r):
        h, l, o = df_split(x)
        ok = ok and o
        sp.append((h, l))
    CA, SA, CB, SB, CG, SG, IR = sp
    irh = abs(IR[0])

    def rnd(v, D):
        nonlocal ok
        a, o = df_round(v, D)
        ok = ok and o
        return a

    def prod(x, y):
        if x[0] == 0 or y[0] == 0:
            return fmul(fmul(x[0], y[0]), irh)
        v = two_sum(*df_mul(df_mul(x, y), IR))
        return rnd(v, fmul(TOL, abs(v[0])))

    def add(x1, y1, z1, x2, y2, neg):
        nonlocal ok
        zz1 = x1[0] == 0 or y1[0] == 0 or z1[0] == 0
        zz2 = x2[0] == 0 or y2[0] == 0
        t1 = df_mul(df_mul(x1, y1), z1)
        t2 = df_mul(x2, y2)
        if neg:
            t2 = (-t2[0], -t2[1])
        if zz1 and zz2:
            return fmul(fadd(t1[0], t2[0]), irh)
        ok = ok and fadd(abs(t1[0]), abs(t2[0])) >= TINY
        v = two_sum(*df_mul(df_add(t1, t2), IR))
        return rnd(v, fmul(TOL, fadd(abs(v[0]), fmul(fadd(abs(t1[0]), abs(t2[0])), irh))))

    A = [prod(CG, CB), add(CG, SB, SA, SG, CA, True), add(CG, SB, CA, SG, SA, False),
         prod(SG, CB), add(SG, SB, SA, CG, CA, False), add(SG, SB, CA, CG, SA, True),
         prod((-SB[0], -SB[1]), (f32(1.0), f32(0.0))), prod(CB, SA), prod(CB, CA)]
    return A, ok


def rows_fp64(ca, sa, cb, sb, cg, sg, r):
    """The definition: R's entries with FP64 products and sums in
    rotation_rows' order, then fl32(fl64(R_i / r))."""
    R = [cg * cb, (cg * sb) * sa - sg * ca, (cg * sb) * ca + sg * sa,
         sg * cb, (sg * sb) * sa + cg * ca, (sg * sb) * ca - cg * sa,
         -sb, cb * sa, cb * ca]
    return [f32(x / r) for x in R]


def _check(angles, r):
    """Every angle triple (alpha, beta, gamma): the double-float rows equal
    the definition's bits where they do not fall back; the number of
    fallbacks."""
    r = float(f32(r))
    inv_r = 1.0 / r
    falls = 0
    for a, b, g in angles:
        cs = (math.cos(a), math.sin(a), math.cos(b), math.sin(b), math.cos(g), math.sin(g))
        A, ok = rows_df(*cs, inv_r)
        if not ok:
            falls += 1
            continue
        want = rows_fp64(*cs, r)
        assert [_bits(x) for x in A] == [_bits(x) for x in want], (a, b, g, A, want)
    return falls


def _grid_angles(name, n_per_level, seed, flags=0):
    w = synth.WORKLOADS[name]
    scan = synth.make_scan(w.scene, 0)[0]
    rg = oracle.make_ranges(w.lo, w.hi, w.ang_lo, w.ang_hi)
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(scan), rg, flags)
    half = 0.0 if flags & oracle.ANGLE_LOWER_EDGE else 0.5
    rng = np.random.default_rng(seed)
    out = []
    for l in range(g.levels):
        N, dp = g.N(l), g.dprime(l)
        total = N[0] * N[1] * N[2]
        idx = range(total) if total <= n_per_level else rng.integers(0, total, n_per_level)
        for t in idx:
            t = int(t)
            ig, q = t % N[2], t // N[2]
            ib, ia = q % N[1], q // N[1]
            out.append(tuple(g.g.ang_lo[i] + (c + half) * dp[i] for i, c in enumerate((ia, ib, ig))))
    return w.r, out


@pytest.mark.parametrize("flags", [0, oracle.ANGLE_LOWER_EDGE])
@pytest.mark.parametrize("name", ["room", "indoor", "outdoor"])
def test_rows_df_on_pose_grids(name, flags):
    """Segment-centre and lower-edge angles (the latter and odd segment
    counts put exact zeros and rounding residues near 1e-17 into the
    tables: both stay on the FP32 path)."""
    r, angles = _grid_angles(name, 500, 7, flags)
    falls = _check(angles, r)
    # fallbacks: entries within 2^-40 of a rounding boundary, and sum entries
    # whose two terms cancel to a few bits (grid angles that nearly satisfy
    # one of R's cancellation identities)
    assert falls <= len(angles) // 200, (falls, len(angles))


def test_rows_df_random_angles():
    rng = np.random.default_rng(11)
    angles = [tuple(x) for x in rng.uniform(-math.pi, math.pi, (4000, 3))]
    falls = _check(angles, 0.2)
    assert falls <= 8
    # and voxel sizes across the supported range
    for r in (0.05, 0.37, 1.0, 3.3):
        assert _check([tuple(x) for x in rng.uniform(-math.pi, math.pi, (300, 3))], r) <= 2


def test_rows_df_special_angles():
    """Exact zeros (sin 0), cos(pi/2) (a residue near 6e-17), entries that
    cancel (gamma near the angle where cos(g) sin(b) sin(a) = sin(g) cos(a)),
    and quarter turns: equal bits or an FP64 fallback, never a wrong value."""
    special = []
    for a in (0.0, 1e-9, math.pi / 2, -math.pi / 2, math.pi, 0.3):
        for b in (0.0, 1e-9, math.pi / 2, -0.05, 0.05):
            for g in (0.0, math.pi / 2, math.pi, -math.pi / 4, 1.0):
                special.append((a, b, g))
    # R1 = cg sb sa - sg ca near zero: tan(g) = sb sa / ca
    for a, b in ((0.04, 0.05), (-0.02, 0.03), (0.5, 0.4)):
        g0 = math.atan2(math.sin(b) * math.sin(a), math.cos(a))
        special += [(a, b, g0 + k * 1e-12) for k in range(-3, 4)]
    _check(special, 0.2)
    _check(special, 1.0)


def test_emulated_fma_is_exact():
    """The emulation's fma rounds the exact value a b + c to the nearest
    float, ties to even (checked against rational arithmetic)."""
    rng = np.random.default_rng(5)
    for _ in range(3000):
        a, b, c = (f32(x) for x in rng.standard_normal(3) * np.ldexp(1.0, rng.integers(-20, 20, 3)))
        exact = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
        got = fma(a, b, c)
        d_got = abs(Fraction(float(got)) - exact)
        for other in (np.nextafter(got, f32(math.inf)), np.nextafter(got, f32(-math.inf))):
            d_o = abs(Fraction(float(other)) - exact)
            assert d_got < d_o or (d_got == d_o and _bits(got) % 2 == 0)


def test_tolerance_decides_the_fallback():
    """With the tolerance raised to the whole half-spacing of the floats every
    case falls back: the fallback test is live."""
    global TOL
    keep = TOL
    try:
        TOL = f32(1.0)
        assert _check([(0.1, 0.2, 0.3), (1.0, -0.5, 2.0)], 0.2) == 2
    finally:
        TOL = keep
