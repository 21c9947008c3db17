"""The exact refinement's two pieces against their integer definitions (bit for bit).

The dense solves track the refinement residual R = E - K B exactly (App. B.2's mixed
precision): P' = P diag(dr) is split into five 8-bit fixed-point slices per row, each
correction into one 8-bit slice per column (integers up to 127), and the tensor cores form
their products as exact integer sums. These tests pin the split to its definition and the
tcgen05 level product to integer arithmetic, including the largest operands (+-128 times
+-127) with signs aligned so that every product of an output entry has one sign: the
1,024-long chunk sums then reach 16,646,144 (the largest the operand bounds allow, below
2^24) and the level sums pass 2^24.
"""
import numpy as np
import pytest
import torch

from paper_2511_04277_gb300 import api

pytestmark = pytest.mark.gpu


def split_reference(P, dr):
    """rg_exact_split's definition in numpy int64: e_i = frexp exponent of the row maximum of
    |P'|, q = rint(P' 2^(39 - e_i)), balanced base-256 digits of q."""
    Pp = P * (dr[None, :] if dr is not None else 1.0)
    n = P.shape[0]
    mx = np.abs(Pp).max(axis=1)
    e = np.where(mx > 0, np.frexp(mx)[1], 0).astype(np.int64)
    q = np.rint(Pp * np.ldexp(1.0, 39 - e)[:, None]).astype(np.int64)
    q[mx == 0] = 0
    d = np.zeros((n, 5, P.shape[1]), np.int64)
    for a in range(4, 0, -1):
        d[:, a] = ((q + 128) & 255) - 128
        q = (q - d[:, a]) >> 8
    d[:, 0] = q
    return d, e


@pytest.mark.parametrize("n,trans,with_dr", [(300, False, True), (300, True, False), (129, False, False),
                                             (517, True, True), (1000, False, True), (70, True, False)])
def test_exact_split_matches_its_definition(rg_ctx, n, trans, with_dr):
    rng = np.random.default_rng(n + 7 * trans)
    # entries spread over 40 binades, signs mixed, some exact zeros and one zero row
    P = rng.uniform(-1, 1, (n, n)) * np.ldexp(1.0, rng.integers(-40, 1, (n, n)))
    P[rng.random((n, n)) < 0.1] = 0.0
    P[5] = 0.0
    dr = rng.uniform(0.05, 0.95, n) if with_dr else None
    P_d = torch.as_tensor(P.T.copy() if trans else P, device="cuda")
    sl, ex = api.exact_split(rg_ctx, P_d, None if dr is None else torch.as_tensor(dr, device="cuda"), trans=trans)
    d_ref, e_ref = split_reference(P, dr)
    sl = sl.cpu().numpy().astype(np.int64)
    np_ = sl.shape[2]
    assert np.array_equal(ex.cpu().numpy(), e_ref)
    assert np.array_equal(sl[:, :, :n], d_ref)
    assert not sl[:, :, n:].any()
    assert np.abs(sl[:, 1:]).max() <= 128 and np.abs(sl[:, 0]).max() <= 128
    # the slices represent P' to 2^(e_i - 40)
    w = np.ldexp(1.0, -8 * np.arange(5))
    rec = np.einsum("iak,a->ik", sl[:, :, :n].astype(np.float64), w) * np.ldexp(1.0, e_ref - 7)[:, None]
    Pp = P * (dr[None, :] if dr is not None else 1.0)
    assert np.all(np.abs(rec - Pp) <= np.ldexp(1.0, e_ref - 40)[:, None])
    del np_


@pytest.mark.parametrize("trans", [False, True])
def test_exact_split_beyond_the_shared_memory_row(rg_ctx, trans):
    """n = 12,300: rows longer than the shared-memory form holds take the two-pass warp form
    (and the transposed form its tiled passes); sampled rows against the definition."""
    n = 12300
    rng = np.random.default_rng(11 + trans)
    P = (rng.uniform(-1, 1, (n, n)) * np.ldexp(1.0, rng.integers(-30, 1, (n, n)))).astype(np.float64)
    dr = rng.uniform(0.05, 0.95, n)
    P_d = torch.as_tensor(P.T.copy() if trans else P, device="cuda")
    sl, ex = api.exact_split(rg_ctx, P_d, torch.as_tensor(dr, device="cuda"), trans=trans)
    rows = np.array([0, 1, 4095, 6150, 12299])
    d_ref, e_ref = split_reference(P[rows], dr)
    assert np.array_equal(ex.cpu().numpy()[rows], e_ref)
    assert np.array_equal(sl[rows].cpu().numpy().astype(np.int64)[:, :, :n], d_ref)
    del P_d, sl


def _ints(rng, shape, extreme=False, top=128, col_signs=None):
    """Random integers in [-top, top]; extreme: +-top; col_signs: +-top with the sign of
    column k from col_signs[k] times a random sign per row (products of two such operands
    share one sign along k)."""
    if col_signs is not None:
        rows = rng.choice(np.array([-1.0, 1.0]), (shape[0], 1))
        return top * rows * col_signs[None, :shape[1]]
    if extreme:
        return rng.choice(np.array([-float(top), float(top)]), shape)
    return rng.integers(-top, top + 1, shape).astype(np.float64)


@pytest.mark.parametrize("M,N,np_,levels,extreme", [
    (300, 257, 256, 5, False),     # ragged tiles, narrow tile widths
    (130, 7, 1024, 3, True),       # every product +-16,256
    (200, 140, 2304, 5, "aligned"),  # full chunks of one sign: sums 16,646,144, two chunks and a short one
    (257, 300, 384, 5, True),      # a level shorter than one chunk
    (4096, 2560, 512, 2, False),   # 128 x 256 tiles
    (2048, 2049, 384, 4, True),    # 128 x 128 tiles with a one-column tail
    (4097, 2600, 512, 3, True),    # CTA pairs (256 x 256): the last pair's odd CTA lies beyond M
    (4000, 2600, 1152, 2, "aligned"),  # CTA pairs, a full chunk of one sign and a short one
])
def test_exact_gemm_is_integer_exact(rg_ctx, M, N, np_, levels, extreme):
    rng = np.random.default_rng(M + N + levels)
    A = np.zeros((M, 5 * np_))
    if extreme == "aligned":
        sk = rng.choice(np.array([-1.0, 1.0]), np_)
        A[:, :levels * np_] = np.concatenate([_ints(rng, (M, np_), col_signs=sk) for _ in range(levels)], axis=1)
        B = _ints(rng, (N, np_), top=127, col_signs=sk)
    else:
        A[:, :levels * np_] = _ints(rng, (M, levels * np_), extreme)
        B = _ints(rng, (N, np_), extreme, top=127)
    A_d = torch.as_tensor(A, device="cuda").to(torch.bfloat16)
    B_d = torch.as_tensor(B, device="cuda").to(torch.bfloat16)
    S = api.tc_gemm_exact(rg_ctx, A_d, B_d, levels).cpu().numpy().astype(np.int64)
    for a in range(levels):
        ref = (A[:, a * np_:(a + 1) * np_] @ B.T).astype(np.int64)   # exact in fp64 (< 2^53)
        assert np.array_equal(S[a], ref), f"level {a}: max diff {np.abs(S[a] - ref).max()}"
