"""Index arithmetic of the CUDA kernels, checked on the CPU over every size they accept.

The kernels replace integer divides by multiply-high divisions and walk packed triangles with
running indices; these tests restate those formulas and compare them with the direct ones for
all orders W <= 128 (the library's limit), so that a change to the ranges or the formulas that
breaks exactness fails here rather than as a wrong shared-memory address on the GPU.
"""
import numpy as np

NT = 256          # threads of the double-float reduction's CTA
MAX_W = 128


def tri(r, c):
    return r * (r + 1) // 2 + c


def fastdiv_magic(d):
    """ceil(2^32 / d) for d >= 2 (FastDiv::magic; d = 1 is special-cased to 0)."""
    return 0 if d <= 1 else (0xFFFFFFFF // d) + 1


def umulhi(a, mag):
    return (a.astype(np.uint64) * np.uint64(mag)) >> np.uint64(32)


def test_fastdiv_magic_is_ceiling():
    for d in range(2, 4097):
        assert fastdiv_magic(d) == -(-(1 << 32) // d)


def test_fastdiv_exact_where_used():
    # the reduction's row / part split: a <= NT, d = trailing-block order 2..255
    a = np.arange(NT + 1, dtype=np.uint64)
    for d in range(2, 256):
        assert np.array_equal(umulhi(a, fastdiv_magic(d)), a // np.uint64(d)), d
    # the Berry kernels' (row, column) split of a W x W index and the eta x W split
    for W in range(2, MAX_W + 1):
        a = np.arange(max(W * W, 64 * W), dtype=np.uint64)
        assert np.array_equal(umulhi(a, fastdiv_magic(W)), a // np.uint64(W)), W


def test_fastdiv_bound_a_times_d_below_2_32():
    # the stated validity bound, probed at its edge for a spread of divisors
    rng = np.random.default_rng(7)
    for d in list(range(2, 300)) + [1000, 4095, 65535]:
        hi = (1 << 32) // d
        a = np.unique(np.concatenate([np.arange(max(0, hi - 2000), hi, dtype=np.int64),
                                      rng.integers(0, hi, 4000)])).astype(np.uint64)
        assert np.array_equal(umulhi(a, fastdiv_magic(d)), a // np.uint64(d)), d


def test_symv_running_indices():
    # thread t takes row r = t mod m and the columns c = part, part + Pp, ...; the lower
    # element (r, c) sits at tri(o + r, o) + c and the mirrored one (c, r) at tri(o + c, o + r),
    # which the kernel advances by (o + c) Pp + Pp (Pp + 1) / 2, that step growing by Pp^2
    for W in list(range(3, 70)) + [96, 127, 128]:
        size = W * (W + 1) // 2
        for i in range(W - 2):
            o, m = i + 1, W - 1 - i
            Pp = NT // m
            for t in range(Pp * m):
                r, part = t % m, t // m
                ilo = tri(o + r, o) + part
                iup = tri(o + part, o + r)
                dup = (o + part) * Pp + (Pp * (Pp + 1)) // 2
                for c in range(part, m, Pp):
                    got = iup if c > r else ilo
                    want = tri(o + c, o + r) if c > r else tri(o + r, o) + c
                    assert got == want and 0 <= got < size
                    ilo += Pp
                    iup += dup
                    dup += Pp * Pp


def test_rank2_index_identity():
    # element (r + 1, c + 1) of the trailing block of step o - 1 (idx = tri(r, c)) sits at
    # idx + r (o + 1) + tri(o + 1, o + 1) of the packed matrix
    for W in list(range(3, 70)) + [96, 127, 128]:
        rows = np.repeat(np.arange(W), np.arange(1, W + 1))
        for i in range(W - 2):
            o, m = i + 1, W - 1 - i
            n1 = m - 1
            idx = np.arange(n1 * (n1 + 1) // 2)
            r = rows[idx]
            c = idx - r * (r + 1) // 2
            got = idx + r * (o + 1) + tri(o + 1, o + 1)
            want = (o + r + 1) * (o + r + 2) // 2 + o + c + 1
            assert np.array_equal(got, want)
            assert got.max(initial=0) < W * (W + 1) // 2
