"""GPU parity of the reduced-precision copies and of the BF16 / FP8 traversal
with FP32 re-rank (compression is orthogonal to the index, Sec. 4.3)."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_same, dev_index, run

pytestmark = pytest.mark.gpu
MV = 16384


def _quant_gpu(X, dtype):
    import torch

    import paper_2408_08933_gb300 as pkg

    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to("cuda:0")
    codes, sc = pkg.quantize(Xd, dtype)
    torch.cuda.synchronize()
    c = codes.cpu().numpy()
    return (c.view(np.uint16) if dtype == "bf16" else c), (None if sc is None else sc.cpu().numpy())


def _edge_rows(d):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((40, d)).astype(np.float32)
    X[0] = 0.0                                  # all-zero row: scale 1
    X[1] = 1e-30                                # tiny values: subnormal codes
    X[2, ::2] = 3.0e38                          # huge values
    X[3] = np.linspace(-1, 1, d).astype(np.float32)
    X[4, 0] = -7.0                              # a negative maximum
    return X


@pytest.mark.parametrize("d", [64, 200])
def test_quantizers_bit_exact(tiny, d):
    X = np.concatenate([_edge_rows(d), np.random.default_rng(d).standard_normal((500, d)).astype(np.float32)])
    got16, _ = _quant_gpu(X, "bf16")
    assert np.array_equal(got16, oracle.quant_bf16(X))
    got8, gs = _quant_gpu(X, "fp8")
    ref8, rs = oracle.quant_e4m3(X)
    assert np.array_equal(gs, rs)
    assert np.array_equal(got8, ref8)


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
@pytest.mark.parametrize("L", [10, 50, 100, 400])
def test_quantized_search_bit_exact(tiny, dtype, L):
    X = tiny["X"]
    if dtype == "bf16":
        codes, sc = oracle.quant_bf16(X), None
    else:
        codes, sc = oracle.quant_e4m3(X)
    idx = dev_index(X, tiny["adj"], tiny["entry"], dtype=dtype, trav=codes.view(np.int16) if dtype == "bf16" else codes,
                    scales=sc, max_visits=MV)
    Q = tiny["Q"]
    ref = oracle.beam_search(X, tiny["adj"], tiny["entry"], Q, 10, L, max_visits=MV, dtype=dtype,
                             Xt=codes, scales=sc)
    assert_same(run(idx, Q, 10, L), ref, f"{dtype} L={L}")
    idx.close()


def test_quantized_recall_close_to_fp32(tiny):
    X, Q, gt = tiny["X"], tiny["Q"], tiny["gt"]
    f32 = oracle.beam_search(X, tiny["adj"], tiny["entry"], Q, 10, 100, max_visits=MV)
    r32 = oracle.recall_at_k(f32[0], gt, 10)
    for dtype in ("bf16", "fp8"):
        codes, sc = (oracle.quant_bf16(X), None) if dtype == "bf16" else oracle.quant_e4m3(X)
        idx = dev_index(X, tiny["adj"], tiny["entry"], dtype=dtype,
                        trav=codes.view(np.int16) if dtype == "bf16" else codes, scales=sc, max_visits=MV)
        got = run(idx, Q, 10, 100)
        idx.close()
        assert abs(oracle.recall_at_k(got[0], gt, 10) - r32) <= 0.005, dtype


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_hand_traced_quantized_case(dtype):
    """The hand-traced case of tests/golden/quant_search_fan.json on the GPU:
    the FP8 scale multiplies once after the fixed-order dot (a tie that one
    rounding decides), the whole final pool is re-ranked in FP32 and ties go
    to the lower id."""
    from conftest import load_golden
    from test_oracle_search import quant_fan_inputs

    g = load_golden("quant_search_fan.json")
    X32, adj, q, fp8, scales, bf16 = quant_fan_inputs(g)
    if dtype == "f32":
        idx = dev_index(X32, adj, g["entry"], max_visits=MV)
    elif dtype == "bf16":
        idx = dev_index(X32, adj, g["entry"], dtype="bf16", trav=bf16.view(np.int16), max_visits=MV)
    else:
        idx = dev_index(X32, adj, g["entry"], dtype="fp8", trav=fp8, scales=scales, max_visits=MV)
    e = g["expect"][dtype]
    for k in (1, 2):
        ids, dist, visits, hops, st = run(idx, q, k, g["L"])
        assert ids[0].tolist() == e[str(k)]["ids"], k
        assert dist[0].tolist() == e[str(k)]["dist"], k
        assert (int(visits[0]), int(hops[0]), int(st[0])) == (e["visits"], e["hops"], 0)
    idx.close()
