"""Reading the packed interception table of a saved layout on the CPU, to
check that its box codes nest: every query the code test of an entry
admits, the code tests of the entry's chunk and super-chunk admit too.

The code of x in a frame (lo, inv) is floor(clamp((x - lo) * inv, -1,
K - 1)) + 1 with each float32 operation rounded on its own (the library's
definition of its 15-bit codes); it is monotone in x, so the values a box's
code test admits on an axis form an interval of float32 values, whose ends
are found here by bisection over the float32 values in order.  A chunk's
entries use a frame of their own, with origin fma(L_c, step, base) rounded
once to float32 and scale inv * 2^e."""
from fractions import Fraction

import numpy as np

K = 32767
CHUNK = 8
ARRAYS = ["kd_nodes", "kd_points", "pos_of_vertex", "row_off", "entries", "edge_rec",
          "face_rec", "edges", "tris", "nb_off", "nb", "chunk_off", "chunks", "nbp",
          "super_off", "supers"]


def read_layout(path):
    """The arrays (uint32) and the global code frame of a saved layout: a
    184-byte header whose last six floats are the frame's origin and scale,
    then per array a uint64 count and that many 4-byte elements."""
    raw = open(path, "rb").read()
    fl = np.frombuffer(raw[108:184], np.float32)
    lo, inv = fl[13:16].copy(), fl[16:19].copy()
    pos, out = 184, {}
    for name in ARRAYS:
        n = int(np.frombuffer(raw[pos:pos + 8], np.uint64)[0])
        out[name] = np.frombuffer(raw[pos + 8:pos + 8 + 4 * n], np.uint32).copy()
        pos += 8 + 4 * n
    return out, lo, inv


def unwords(w):
    """(..., 3) code words -> lower codes (..., 3), upper codes (..., 3)"""
    w = w.astype(np.int64)
    lo = np.stack([w[..., 0] & 0xFFFF, w[..., 0] >> 16, w[..., 1] & 0xFFFF], -1)
    hi = K - np.stack([w[..., 1] >> 16, w[..., 2] & 0xFFFF, w[..., 2] >> 16], -1)
    return lo, hi


def _key(x):
    """float32 -> int64 keys in the order of the values (-0 and +0 alike)"""
    i = np.asarray(x, np.float32).view(np.int32).astype(np.int64)
    return np.where(i >= 0, i, -(i & 0x7FFFFFFF))


def _val(k):
    k = np.asarray(k, np.int64)
    return np.where(k >= 0, k, (-k) | 0x80000000).astype(np.uint32).view(np.float32)


def code(x, lo, inv):
    d = (np.asarray(x, np.float32) - np.asarray(lo, np.float32)).astype(np.float32)
    with np.errstate(over="ignore", invalid="ignore"):
        t = (d * np.asarray(inv, np.float32)).astype(np.float32)
    t = np.minimum(np.maximum(t, np.float32(-1)), np.float32(K - 1))
    return np.floor(t).astype(np.int64) + 1


LOW, HIGH = int(_key(np.float32(-3e38))), int(_key(np.float32(3e38)))


def first_key_at_least(c, lo, inv):
    """Key of the smallest float32 x in [-3e38, 3e38] whose code is >= c
    (c >= 1; the code of -3e38 is 0 and that of 3e38 is K)."""
    a = np.full(np.shape(c), LOW, np.int64)
    b = np.full(np.shape(c), HIGH, np.int64)
    while True:
        open_ = b - a > 1
        if not open_.any():
            return b
        m = (a + b) // 2
        ok = code(_val(m), lo, inv) >= c
        b = np.where(open_ & ok, m, b)
        a = np.where(open_ & ~ok, m, a)


def admitted(L, H, lo, inv):
    """Keys of the first and last float32 values whose code lies in [L, H]
    (L = 0: no lower end; H = K: no upper end)."""
    L, H = np.asarray(L), np.asarray(H)
    first = np.where(L > 0, first_key_at_least(np.maximum(L, 1), lo, inv), LOW - 1)
    last = np.where(H < K, first_key_at_least(np.minimum(H + 1, K), lo, inv) - 1, HIGH + 1)
    return first, last


def fma_f32(a, b, c):
    """a * b + c rounded once to float32 (ties to even), from exact rationals."""
    exact = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    f = np.float32(float(exact))
    best = None
    for g in (np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))):
        err = abs(Fraction(float(g)) - exact)
        even = int(np.float32(g).view(np.uint32)) % 2 == 0
        if best is None or err < best[0] or (err == best[0] and even and not best[2]):
            best = (err, g, even)
    return np.float32(best[1])


def check_codes_nest(arr, glo, ginv):
    """Every entry's admitted interval on each axis lies inside its chunk's,
    every chunk's inside its super-chunk's; returns the number of entries."""
    row_off, chunk_off, super_off = arr["row_off"], arr["chunk_off"], arr["super_off"]
    nv = len(row_off) - 1
    ent = arr["entries"].reshape(-1, 4)
    chk = arr["chunks"].reshape(-1, 4)
    sup = arr["supers"].reshape(-1, 4)
    assert len(chunk_off) == nv + 1 and len(super_off) == nv + 1
    # the chunk and super-chunk of every entry and chunk
    e_chunk = np.empty(len(ent), np.int64)
    c_super = np.empty(len(chk), np.int64)
    for p in range(nv):
        r0, r1 = int(row_off[p]), int(row_off[p + 1])
        c0, c1 = int(chunk_off[p]), int(chunk_off[p + 1])
        s0, s1 = int(super_off[p]), int(super_off[p + 1])
        assert c1 - c0 == -(-(r1 - r0) // CHUNK) and s1 - s0 == -(-(c1 - c0) // CHUNK)
        e_chunk[r0:r1] = c0 + np.arange(r1 - r0) // CHUNK
        c_super[c0:c1] = s0 + np.arange(c1 - c0) // CHUNK
    cl, ch = unwords(chk[:, :3])
    sl, sh = unwords(sup[:, :3])
    el, eh = unwords(ent[:, 1:])
    # super-chunks hold their chunks (one frame: compare the codes)
    assert (sl[c_super] <= cl).all() and (ch <= sh[c_super]).all()
    glo = np.asarray(glo, np.float32)
    ginv = np.asarray(ginv, np.float32)
    step = (np.float32(1) / ginv).astype(np.float32)
    base = (glo - step).astype(np.float32)
    for d in range(3):
        # the entry frame of every chunk on this axis
        expo = (chk[:, 3].astype(np.int64) >> (8 * d)) & 0xFF
        c_lo = np.array([fma_f32(x, step[d], base[d]) for x in cl[:, d]], np.float32)
        c_inv = (ginv[d] * np.ldexp(np.float32(1), expo).astype(np.float32)).astype(np.float32)
        e_first, e_last = admitted(el[:, d], eh[:, d], c_lo[e_chunk], c_inv[e_chunk])
        assert (e_first <= e_last).all(), d
        k_first, k_last = admitted(cl[:, d], ch[:, d], glo[d], ginv[d])
        assert (k_first[e_chunk] <= e_first).all() and (e_last <= k_last[e_chunk]).all(), d
    return len(ent)
