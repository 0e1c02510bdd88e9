"""The split-precision reading of the tensor-core FC forms, checked in FP64
with an emulation of BF16 round-to-nearest-even (no GPU).

With Z = H + L, H = bf16(Z) and L = bf16(Z - H), the three-product Gram
matrix H H^T + H L^T + L H^T leaves out L L^T. That term, like the rounding of
L itself, is about 2^-16 of G (far above FP32 rounding), so the BF16x3 form
reaches a few 1e-6 of the normalising scale sqrt(G_kk G_jj), well inside the
1e-4 FC tolerance; the single BF16 form (H H^T alone) is two to three orders
coarser. The three products are symmetric in exact arithmetic."""
import numpy as np


def _bf16(x):
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def test_bf16_split_gram_error():
    rng = np.random.default_rng(1)
    N, T = 68, 500
    Z = (1e-4 * rng.standard_normal((N, T))).astype(np.float32)   # a shifted rate series, kHz
    H = _bf16(Z)
    L = _bf16(Z.astype(np.float64) - H.astype(np.float64))
    Zd, Hd, Ld = (a.astype(np.float64) for a in (Z, H, L))
    G = Zd @ Zd.T
    scale = np.sqrt(np.outer(np.diag(G), np.diag(G)))
    G3 = Hd @ Hd.T + Hd @ Ld.T + Ld @ Hd.T
    G1 = Hd @ Hd.T
    err3 = (np.abs(G3 - G) / scale).max()
    err1 = (np.abs(G1 - G) / scale).max()
    ll = (np.abs(Ld @ Ld.T) / scale).max()
    assert 1e-7 < ll < 2e-5            # about 2^-16, far above FP32 rounding (6e-8)
    assert err3 < 2e-5                 # a few 1e-6
    assert err1 > 100 * err3           # the single form is far coarser
    assert np.allclose(G3, G3.T, rtol=0, atol=1e-12 * np.abs(G).max())
    # the split itself: H carries 8 significant bits, |L| <= 2^-8 |Z|
    assert (np.abs(Zd - Hd) <= 2.0 ** -8 * np.abs(Zd) + 1e-30).all()
