"""The FP32 cutoff screen of the W-form reconstruction (CPU check of its
error bound, no GPU).  The kernel forms FP32 coefficients a32 = G32 dh from
FP32-rounded matrix rows G32 and FP32 differences dh (on the FP64 path a
truncating FP64 -> FP32 conversion of d = U_s - U_0), sums their squares in
FP32, and bounds |beta32 - beta| by

  eb = (m + 2) u beta32 + E (2 sqrt(beta32) + E),  E = 1.0001 (n + 7) u e_abs,

with u = 2^-24 and e_abs = sum_s colsum_s |dh_s|, colsum_s = sum_l |G_ls|
(the rigorous bound of the screen; the cutoff decision is taken from the FP32
values only when chi is provably on one side of C_T).  Here that FP32
arithmetic is emulated step by step in numpy on random matrices and
differences, including differences that cancel, and the exact beta = |G d|^2
in FP64 must lie within eb of beta32 every time."""
import numpy as np
import pytest

U32 = 2.0 ** -24


def trunc32(x):
    """FP64 -> FP32 rounding toward zero (the kernel's integer conversion),
    for magnitudes in the normal FP32 range."""
    b = np.asarray(x, dtype=np.float64).view(np.uint64)
    b = b & ~np.uint64((1 << 29) - 1)  # drop the 29 low significand bits
    return b.view(np.float64).astype(np.float32)


def fmaf(a, b, c):
    """FP32 fused multiply-add: the product of two FP32 numbers is exact in
    FP64, one rounding to FP32 at the end."""
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def screen(G64, d, truncate):
    m, n = G64.shape
    G32 = G64.astype(np.float32)
    dh = trunc32(d) if truncate else d.astype(np.float32)
    colsum = np.abs(G64).sum(axis=0).astype(np.float32)
    a32 = np.zeros(m, dtype=np.float32)
    e_abs = np.float32(0.0)
    for s in range(n):
        for l in range(m):
            a32[l] = fmaf(G32[l, s], dh[s], a32[l])
        e_abs = fmaf(colsum[s], np.float32(abs(dh[s])), e_abs)
    b32 = np.float32(0.0)
    for l in range(m):
        b32 = fmaf(a32[l], a32[l], b32)
    E = np.float32((n + 7) * U32 * float(e_abs) * 1.0001)
    eb = (m + 2) * U32 * float(b32) + float(E) * (2.0 * np.sqrt(float(b32)) + float(E))
    beta = float(np.sum((G64 @ d) ** 2))
    return float(b32), beta, eb


@pytest.mark.parametrize("truncate", [True, False], ids=["fp64-path", "pair-path"])
@pytest.mark.parametrize("m,n", [(20, 42), (14, 30), (5, 12)])
def test_screen_bound_holds(m, n, truncate):
    rng = np.random.default_rng(100 * m + n + int(truncate))
    worst = 0.0
    for trial in range(300):
        # least-squares-like rows: mixed signs, magnitudes over four decades
        G = rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-1, 3, (m, 1))
        kind = trial % 3
        if kind == 0:    # smooth data: differences of one sign and size
            d = rng.uniform(0.5, 1.5, n) * 10.0 ** rng.uniform(-6, 1)
        elif kind == 1:  # a jump: a few large differences among small ones
            d = rng.standard_normal(n) * 1e-4
            d[rng.choice(n, 3, replace=False)] += rng.standard_normal(3) * 5.0
        else:            # differences in the null space's neighbourhood: G d cancels
            d = rng.standard_normal(n)
            q, _ = np.linalg.qr(G.T)
            d = d - q @ (q.T @ d) + 1e-7 * rng.standard_normal(n)
        b32, beta, eb = screen(G, d, truncate)
        assert abs(b32 - beta) <= eb, (trial, b32, beta, eb)
        worst = max(worst, abs(b32 - beta) / eb if eb > 0 else 0.0)
    assert worst > 1e-4  # the bound is exercised, not vacuous


def test_truncation_error():
    """The integer conversion's relative error is below 2u = 2^-23, toward zero."""
    x = np.random.default_rng(7).standard_normal(100000) * 10.0 ** np.random.default_rng(8).uniform(-30, 30, 100000)
    t = trunc32(x).astype(np.float64)
    assert np.all(np.abs(t) <= np.abs(x))
    assert np.max(np.abs(t - x) / np.abs(x)) < 2.0 ** -23
