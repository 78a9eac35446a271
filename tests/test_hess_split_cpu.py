"""The arithmetic of the tensor-core Hessian, on the CPU: each entry of J (the
per-event gradients d_i of ln I, float32) is split into three BF16 terms
d = b1 + b2 + b3 by round-to-nearest-even, and H = J^T J is assembled from
the products D = [b1; b2; b3] [b1; b2]^T (rows 0..R-1 b1, R..2R-1 b2,
2R..3R-1 b3) as
  H_pq = T[p][q] + T[R + p][q] + T[2R + p][q] + T[2R + q][p],
  T[m][q] = D[m][q] + D[m][R + q] for m < 2R, D[m][q] otherwise.
Checked against J^T J in FP64: the split is exact but for the rounding of
the third term, and the dropped products (b2 b3, b3 b2, b3 b3) are below
2^-23 of |d_p d_q|. A mistake in the row offsets or a missing transposed b3
term fails by many orders of magnitude.
"""
import numpy as np


def bf16_rn(x):
    """float32 -> the nearest BF16 value (ties to even), as float32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def split3(J):
    b1 = bf16_rn(J)
    r1 = (J - b1).astype(np.float32)
    b2 = bf16_rn(r1)
    r2 = (r1 - b2).astype(np.float32)
    return b1, b2, bf16_rn(r2)


def assemble(J):
    """H from the BF16 terms through the tensor-core products (FP64 sums)."""
    n, R = J.shape
    b1, b2, b3 = split3(J)
    A = np.concatenate([b1, b2, b3], axis=1).astype(np.float64)   # rows of the K-major tile
    B = np.concatenate([b1, b2], axis=1).astype(np.float64)
    D = A.T @ B                                                  # [3R, 2R]
    T = D[:, :R].copy()
    T[:2 * R] += D[:2 * R, R:]
    Hraw = T[:R] + T[R:2 * R] + T[2 * R:] + T[2 * R:].T
    # entries p <= q, mirrored (as the finalize writes both halves)
    return np.triu(Hraw) + np.triu(Hraw, 1).T


def sample_J(n, R, seed):
    rng = np.random.default_rng(seed)
    # magnitudes spread over several decades per event, as |A| / |S| varies
    scale = np.exp(rng.normal(0.0, 2.0, size=(n, 1)))
    return (rng.normal(size=(n, R)) * scale).astype(np.float32)


def test_split_is_exact_but_for_the_third_rounding():
    J = sample_J(20000, 40, 1)
    b1, b2, b3 = split3(J)
    for b in (b1, b2, b3):
        assert np.all((b.view(np.uint32) & 0xFFFF) == 0)   # representable in BF16
    resid = J.astype(np.float64) - (b1.astype(np.float64) + b2 + b3)
    assert np.all(np.abs(resid) <= 2.0 ** -24 * np.abs(J.astype(np.float64)))


def test_assembled_hessian_matches_jtj():
    for R, seed in ((8, 2), (24, 3), (40, 4)):
        J = sample_J(5000, R, seed)
        Jd = J.astype(np.float64)
        H_ref = Jd.T @ Jd
        H = assemble(J)
        assert np.array_equal(H, H.T)
        # per entry: the third term's rounding (2^-24 |d|, twice) and the
        # dropped products (2^-16 2^-8 twice + 2^-32) against sum |d_p| |d_q|
        bound = 2.0 ** -21 * (np.abs(Jd).T @ np.abs(Jd))
        assert np.all(np.abs(H - H_ref) <= bound)


def test_wrong_assembly_is_caught():
    """The same check fails when the transposed b3 term is left out or the
    b2 rows are taken at the wrong offset."""
    J = sample_J(5000, 24, 5)
    Jd = J.astype(np.float64)
    H_ref = Jd.T @ Jd
    bound = 2.0 ** -21 * (np.abs(Jd).T @ np.abs(Jd))
    n, R = J.shape
    b1, b2, b3 = split3(J)
    A = np.concatenate([b1, b2, b3], axis=1).astype(np.float64)
    B = np.concatenate([b1, b2], axis=1).astype(np.float64)
    D = A.T @ B
    T = D[:, :R].copy()
    T[:2 * R] += D[:2 * R, R:]
    no_transpose = T[:R] + T[R:2 * R] + T[2 * R:]
    assert not np.all(np.abs(no_transpose - H_ref) <= bound)
    Tw = D[:, :R].copy()
    Tw[:2 * R] += D[:2 * R, :R]          # b1 columns twice instead of b1 + b2
    wrong_cols = Tw[:R] + Tw[R:2 * R] + Tw[2 * R:] + Tw[2 * R:].T
    assert not np.all(np.abs(wrong_cols - H_ref) <= bound)
