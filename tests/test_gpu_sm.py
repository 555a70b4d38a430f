"""Sherman-Morrison inverse update on the GPU (blip_sm_update) against the
FP64 oracle (the same formula on the same FP32 inputs), under an FP32
rounding bound, plus the identity D' Dinv' ~ I against the updated matrix."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
U = 2.0 ** -24


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_1121_gb300 as pb
    return pb


@pytest.mark.parametrize("n", [1, 5, 33, 96, 257, 768, 1024, 1100])
def test_sm_update_matches_oracle(pb, n):
    rng = np.random.default_rng(n)
    W = 5
    Ds = [rng.normal(size=(n, n)) + 3.0 * np.sqrt(n) * np.eye(n) for _ in range(W)]
    dinv32 = np.stack([np.linalg.inv(D) for D in Ds]).astype(np.float32)
    rows = rng.normal(size=(W, n)).astype(np.float32)
    cols = np.array([0, n - 1, -1, n // 2, (7 % n)], dtype=np.int32)
    d = torch.from_numpy(dinv32.copy()).cuda()
    pb.sm_update(d, torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda())
    got = d.cpu().numpy().astype(np.float64)
    for w in range(W):
        j = int(cols[w])
        if j < 0:
            assert np.array_equal(got[w], dinv32[w])          # untouched
            continue
        ref, ww = oracle.sherman_morrison.sm_update(dinv32[w], rows[w], j)
        absD, rank1, S, _ = oracle.sherman_morrison.sm_update_terms(dinv32[w], rows[w], j)
        colj = np.abs(dinv32[w][:, j].astype(np.float64))
        # FP32: w_k carries up to n U S_k, the division and the FMA a few U
        bound = 4 * U * (absD + rank1) + colj[:, None] * (
            n * U * S[None, :] / abs(ww[j]) + np.abs(ww - (np.arange(n) == j))[None, :]
            * n * U * S[j] / ww[j] ** 2)
        assert (np.abs(got[w] - ref) <= bound + 1e-30).all()
        # and it is the inverse of the updated matrix (FP32-level accuracy)
        D2 = Ds[w].copy()
        D2[j] = rows[w]
        assert np.abs(D2 @ got[w] - np.eye(n)).max() < 1e-4


def test_sm_update_rejects_bad_arguments(pb):
    L = pb.lib()
    assert L.blip_sm_update(1, 0, None, None, None, None, None) == -1
    assert L.blip_sm_update(0, 4, None, None, None, None, None) == 0
    assert L.blip_sm_update(2, 4, None, None, None, None, None) == -1
