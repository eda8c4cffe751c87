"""The warp-parallel application of the previous Givens rotations to a new
Hessenberg column (givens_core): the carry a_{i+1} = -conj(s_i) a_i + c_i h_{i+1}
is an affine map per rotation; 32 lanes compose the maps of their ranges of
i, an inclusive shuffle scan (lane l combines with lane l - d, d = 1, 2, 4, ...)
composes the ranges below each lane, the exclusive prefix gives each lane its
incoming carry, and the lanes walk their ranges.  Written out in numpy with
the kernel's lane partition and composition order, against the serial
rotation sequence, for columns shorter than, equal to and longer than a warp.
Plain numpy, no GPU."""
import numpy as np
import pytest


def serial(h, c, s):
    col = h.copy()
    j = len(h) - 1
    for i in range(j):
        a, b = col[i], col[i + 1]
        col[i] = c[i] * a + s[i] * b
        col[i + 1] = -np.conj(s[i]) * a + c[i] * b
    return col


def warp_scan(h, c, s):
    j = len(h) - 1
    per = (j + 31) // 32
    lanes = range(32)
    rng = [(min(j, l * per), min(j, min(j, l * per) + per)) for l in lanes]
    A = np.ones(32, complex)
    B = np.zeros(32, complex)
    for l in lanes:                            # this lane's maps composed: M_{e-1} o ... o M_b
        b0, e = rng[l]
        for i in range(b0, e):
            Ai, Bi = -np.conj(s[i]), c[i] * h[i + 1]
            B[l] = Ai * B[l] + Bi
            A[l] = Ai * A[l]
    d = 1
    while d < 32:                              # inclusive scan, shfl_up semantics
        Ao, Bo = A.copy(), B.copy()
        for l in lanes:
            if l >= d:
                B[l] = A[l] * Bo[l - d] + B[l]
                A[l] = A[l] * Ao[l - d]
        d *= 2
    col = np.zeros(j + 1, complex)
    carry = np.zeros(32, complex)
    for l in lanes:                            # exclusive prefix, then the walk
        Ae, Be = (1.0, 0.0) if l == 0 else (A[l - 1], B[l - 1])
        a = Ae * h[0] + Be
        b0, e = rng[l]
        for i in range(b0, e):
            col[i] = s[i] * h[i + 1] + c[i] * a
            a = -np.conj(s[i]) * a + c[i] * h[i + 1]
        carry[l] = a
    last = (j - 1) // per if j > 0 else 0
    col[j] = carry[last] if j > 0 else h[0]
    return col


@pytest.mark.parametrize("j", [0, 1, 5, 31, 32, 33, 64, 95, 119])
def test_scan_equals_serial_rotations(j):
    r = np.random.default_rng(j)
    h = r.standard_normal(j + 1) + 1j * r.standard_normal(j + 1)
    th = r.random(j) * np.pi / 2
    ph = r.random(j) * 2 * np.pi
    c = np.cos(th)
    s = np.sin(th) * np.exp(1j * ph)
    ref = serial(h, c, s)
    got = warp_scan(h, c, s)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
