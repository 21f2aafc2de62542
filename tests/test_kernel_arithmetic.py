"""The integer and floating-point identities the scoring kernel relies on,
checked on the CPU: the 4-bit child counters and the brick planes' child
masks, the bit pattern of
a floored level key, the folded index constant of clamp-free runs, and the
FP32 bound of the per-run inside test (emulated with FP32 arithmetic, the
tightest point placed on the bound)."""
import math
import struct
from fractions import Fraction

import numpy as np

KB = 0x4B400000   # bit pattern of 1.5 * 2^23


def _lut_entry(v):
    # the scoring kernel's child counter increment (child_lut_entry): child
    # i = jx + 2 jy + 4 jz of the 8-bit mask v at bits 4 i .. 4 i + 3
    out = 0
    for i in range(8):
        out |= ((v >> i) & 1) << (4 * i)
    return out


def test_child_counter_words():
    """A scoring thread counts at most 7 points of a task (a 1568-point chunk
    over 224 scoring threads): summing their counter increments never
    carries between 4-bit counters, the even and the odd children's
    counters spread to bytes (acc & 0x0F0F0F0F, (acc >> 4) & 0x0F0F0F0F) sum
    over a warp's 32 lanes without a carry between bytes (at most 224), and
    byte q of the even word holds child 2 q, of the odd word child 2 q + 1;
    then seven warps' bytes 0, 2 and 1, 3 summed in 16-bit fields stay
    below 2^16.  Random mixes of masks and the all-ones worst case."""
    assert 1568 // 224 == 7 and 1568 % 224 == 0
    rng = np.random.default_rng(1)
    for trial in range(300):
        warps_ev, warps_od = [], []
        counts = np.zeros(8, np.int64)
        for w in range(7):
            ev = od = 0
            for lane in range(32):
                n = 7 if trial == 0 else int(rng.integers(0, 8))
                vs = [255] * n if trial == 0 else [int(x) for x in rng.integers(0, 256, n)]
                acc = sum(_lut_entry(v) for v in vs)
                assert acc < 1 << 32
                for i in range(8):
                    assert (acc >> (4 * i)) & 15 == sum((v >> i) & 1 for v in vs)
                    counts[i] += sum((v >> i) & 1 for v in vs)
                ev += acc & 0x0F0F0F0F
                od += (acc >> 4) & 0x0F0F0F0F
            assert ev < 1 << 32 and od < 1 << 32
            for q in range(4):   # no carry between bytes: each byte is its own sum
                assert (ev >> (8 * q)) & 255 <= 224 and (od >> (8 * q)) & 255 <= 224
            warps_ev.append(ev)
            warps_od.append(od)
        for k, words in ((0, warps_ev), (1, warps_od)):
            lo = sum(x & 0x00FF00FF for x in words)
            hi = sum((x >> 8) & 0x00FF00FF for x in words)
            assert lo < 1 << 32 and hi < 1 << 32
            got = {k + 0: lo & 0xFFFF, k + 2: hi & 0xFFFF, k + 4: lo >> 16, k + 6: hi >> 16}
            for i, c in got.items():
                assert c == counts[i], (trial, i)


def test_plane_mask_takes_the_children_bits():
    """The brick layouts' plane words hold children jx + 5 jy of the z = 0 and
    z = 1 planes at bits {0, 1, 5, 6}; their 8-bit child mask has child
    jx + 2 jy + 4 jz at bit jx + 2 jy + 4 jz, for every pair of planes
    (other bits of the words ignored)."""
    def planes_mask(w0, w1):
        return (w0 & 3) | ((w0 >> 3) & 0xC) | ((w1 & 3) << 4) | ((w1 << 1) & 0xC0)
    rng = np.random.default_rng(2)
    for _ in range(20000):
        w0, w1 = (int(x) for x in rng.integers(0, 1 << 32, 2, dtype=np.uint64))
        want = 0
        for i in range(8):
            jx, jy, jz = i & 1, (i >> 1) & 1, i >> 2
            w = w1 if jz else w0
            want |= ((w >> (jx + 5 * jy)) & 1) << i
        assert planes_mask(w0, w1) == want


def test_floored_key_bit_pattern():
    """For C = 1.5 * 2^23 + d (|d| < 2^21) and |q / 2^m| < 2^18, the value
    q 2^-m + C lies in [2^23, 2^24) where FP32 spacing is 1, so rounding down
    gives its floor exactly and the bit pattern is KB + floor(q / 2^m) + d."""
    rng = np.random.default_rng(0)
    for _ in range(3000):
        m = int(rng.integers(0, 12))
        q = float(np.float32(rng.uniform(-(2.0 ** 18), 2.0 ** 18) * 2.0 ** m / 4))
        d = int(rng.integers(-(2 ** 20), 2 ** 20))
        x = Fraction(q) / 2 ** m + Fraction(3 * 2 ** 22 + d)
        assert 2 ** 23 <= x < 2 ** 24
        rd = math.floor(x)
        bits = struct.unpack("<I", struct.pack("<f", float(rd)))[0]
        assert bits == KB + math.floor(Fraction(q) / 2 ** m) + d


def test_folded_index_constant():
    """A run's base index of a point, ((bx ny + by) nz + bz) mod 2^32 with the
    offset-free patterns b = KB + k (k = floor(q / 2^m), any sign), plus a
    task's delta = ((ox ny + oy) nz + oz - KB (ny nz + nz + 1)) mod 2^32 (any
    signs of o), equals the byte index ((kx + ox) ny + (ky + oy)) nz + (kz + oz)
    of key k + o whenever k + o lies in the grid (index below 2^31)."""
    rng = np.random.default_rng(1)
    M = 1 << 32
    for _ in range(3000):
        ny, nz = int(rng.integers(2, 4000)), int(rng.integers(2, 4000))
        nx = int(rng.integers(2, max(3, (1 << 31) // (ny * nz))))
        r = [int(rng.integers(0, n)) for n in (nx, ny, nz)]          # the key in the grid
        o = [int(rng.integers(-(1 << 21), 1 << 21)) for _ in range(3)]   # the task's offset
        k = [r[i] - o[i] for i in range(3)]                              # the rotated point's key
        assert all(abs(x) < 1 << 22 for x in k)
        b = [(KB + x) % M for x in k]
        base = ((b[0] * ny + b[1]) % M * nz + b[2]) % M
        delta = ((o[0] * ny + o[1]) * nz + o[2] - KB * (ny * nz + nz + 1)) % M
        assert (base + delta) % M == (r[0] * ny + r[1]) * nz + r[2]


def _rot(ang, r):
    ca, sa = np.cos(ang), np.sin(ang)
    Rx = np.array([[1, 0, 0], [0, ca[0], -sa[0]], [0, sa[0], ca[0]]])
    Ry = np.array([[ca[1], 0, sa[1]], [0, 1, 0], [-sa[1], 0, ca[1]]])
    Rz = np.array([[ca[2], -sa[2], 0], [sa[2], ca[2], 0], [0, 0, 1]])
    return (Rz @ Ry @ Rx / r).astype(np.float32)


def test_inside_bound_has_no_false_positive():
    """The run's inside test (FP32 corner products widened by 2e-6 of
    sum |A| max |x|) never admits a run with a point whose FP32 key leaves
    [0, rmax + 1], including runs placed with the extreme point exactly on
    either bound."""
    f32 = np.float32
    rng = np.random.default_rng(2)
    admitted = 0
    for _ in range(1500):
        r = float(rng.choice([0.05, 0.2, 0.5, 1.0]))
        m = int(rng.integers(0, 8))
        A = _rot(rng.uniform(-np.pi, np.pi, 3) * rng.choice([1.0, 0.05]), r)
        n = int(rng.integers(1, 1569))
        P = (rng.uniform(-1, 1, (n, 3)) * rng.uniform(0.1, 60.0, 3) + rng.uniform(-20, 20, 3)).astype(f32)
        lo3, hi3 = P.min(0), P.max(0)
        q = ((A[:, 0][None] * P[:, 0:1]).astype(f32) + (A[:, 1][None] * P[:, 1:2]).astype(f32)).astype(f32)
        q = (q + (A[:, 2][None] * P[:, 2:3]).astype(f32)).astype(f32)
        fl = np.floor(q.astype(np.float64) * 2.0 ** -m)
        rmax = rng.integers(10, 5000, 3)
        s = f32(2.0 ** -m)
        for mode in range(3):
            o = (-fl.min(0) if mode == 0 else (rmax + 1) - fl.max(0) if mode == 1
                 else rng.integers(-100, 5000, 3).astype(np.float64))
            inside = True
            for i in range(3):
                qlo = qhi = mag = f32(0)
                for k in range(3):
                    a = A[i, k]
                    p1, p2 = f32(a * lo3[k]), f32(a * hi3[k])
                    qlo, qhi = f32(qlo + min(p1, p2)), f32(qhi + max(p1, p2))
                    mag = f32(mag + f32(abs(a) * max(abs(lo3[k]), abs(hi3[k]))))
                marg = f32(f32(f32(2e-6) * mag) + f32(1e-30))
                oi = f32(o[i])
                inside &= bool(f32(np.floor(f32(f32(qlo - marg) * s))) + oi >= 0)
                inside &= bool(f32(np.floor(f32(f32(qhi + marg) * s))) + oi <= f32(rmax[i]) + f32(1))
            if inside:
                admitted += 1
                keys = fl + o[None, :]
                assert keys.min() >= 0 and np.all(keys <= (rmax + 1)[None, :])
    assert admitted > 100


def test_exponent_range_test():
    """The FP32 rounding of R / r takes its fast path when |q| lies in
    [2^-120, 2^120); testing the biased exponent e as the unsigned
    (e - 903) mod 2^32 < 240 is the same test for every double, signed
    zeros, subnormals, both bounds, infinities and NaN included."""
    def by_value(q):
        return abs(q) >= 2.0 ** -120 and abs(q) < 2.0 ** 120

    def by_bits(q):
        e = (struct.unpack("<Q", struct.pack("<d", q))[0] >> 52) & 0x7FF
        return (e - (1023 - 120)) % (1 << 32) < 240

    edge = [0.0, 5e-324, 2.0 ** -1022, 2.0 ** -120, 2.0 ** 120, 1.0, 1e300, math.inf, math.nan]
    edge += [np.nextafter(v, d) for v in (2.0 ** -120, 2.0 ** 120) for d in (0.0, math.inf)]
    rng = np.random.default_rng(3)
    vals = edge + list(np.ldexp(rng.uniform(1, 2, 20000), rng.integers(-1074, 1024, 20000)))
    for v in vals:
        for q in (float(v), -float(v)):
            assert by_value(q) == by_bits(q), q


def test_edge_key_clamp_from_shared_patterns():
    """Slices near the grid's edge share their run's offset-free patterns
    b = KB + k (|k| < 2^19) and add o - KB (|o| <= 2^21) mod 2^32 per axis:
    the sum is the relative key k + o when that is in [0, rmax + 1], and any
    key outside (negative keys wrap past 2^31) is clamped by min to rmax + 1,
    the empty key past the box -- the same key as clamping k + o directly."""
    rng = np.random.default_rng(3)
    M = 1 << 32
    for _ in range(20000):
        k = int(rng.integers(-(1 << 19) + 1, 1 << 19))
        o = int(rng.integers(-(1 << 21), (1 << 21) + 1))
        rmax = int(rng.integers(0, 1 << 20))
        if rng.random() < 0.5:   # keys near the box
            o = int(rng.integers(-k - 3, -k + rmax + 4))
        r = ((KB + k) % M + (o - KB) % M) % M
        got = min(r, rmax + 1)
        key = k + o
        want = key if 0 <= key <= rmax + 1 else rmax + 1
        assert got == want, (k, o, rmax)
