"""PQ distance tables built on the tensor cores (tcgen05) against the
oracle's FP32 tables (§4.1), and the reduced-precision search fed by them."""
import numpy as np
import pytest

import oracle
from tests import cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2401_11324_gb300 as bang  # noqa: E402


def _workload(which):
    if which == "u8":
        return cases.clustered(n=20_000, nq=300, ncomp=8)
    if which == "f32":
        return cases.config1()
    if which == "i8":
        return cases.clustered(n=8_000, nq=40, ncomp=4, dtype="i8", d=100, M=30, R=40,
                               centre="uniform100")
    return cases.clustered(n=5_000, nq=30, ncomp=4, dtype="f32", d=200, M=50, R=48,
                           centre="uniform255")


def _tc(w, Q, bf16, tf32=False):
    ix = bang.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], w["M"])
    q = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    out = torch.empty((len(Q), w["M"], 256), device="cuda",
                      dtype=torch.bfloat16 if bf16 else torch.float32)
    bang.bang_pq_tables(ix.h, q, len(Q), out, (1 if bf16 else 0) | (2 if tf32 else 0))
    torch.cuda.synchronize()
    ix.close()
    return out.float().cpu().numpy()


@pytest.mark.parametrize("which", ["u8", "f32", "i8", "f32wide"])
def test_tensor_core_tables_match_fp32_oracle(which):
    w = _workload(which)
    Q = w["queries"]
    M, d = w["M"], Q.shape[1]
    T = _tc(w, Q, bf16=False)
    off = oracle.chunk_offsets(d, M)
    cb = w["codebook"].astype(np.float64)
    for qi in range(0, len(Q), max(1, len(Q) // 25)):
        ref = oracle.adc_table(Q[qi].astype(np.float32), M, w["codebook"]).astype(np.float64)
        qf = Q[qi].astype(np.float64)
        for s in range(M):
            o, ds = off[s], off[s + 1] - off[s]
            C = cb[256 * o: 256 * o + 256 * ds].reshape(256, ds)
            scale = (qf[o:o + ds] ** 2).sum() + (C ** 2).sum(1)      # size of the cancelling terms
            err = np.abs(T[qi, s] - ref[s])
            assert (err <= 4e-6 * scale + 2e-3).all(), (which, qi, s, err.max())
    Tb = _tc(w, Q, bf16=True)
    rounded = torch.from_numpy(T).to(torch.bfloat16).float().numpy()
    assert (np.abs(Tb - rounded) <= 2.0 ** -7 * np.abs(rounded) + 1e-3).all()


def test_bf16_search_on_tensor_core_tables():
    w = cases.clustered(n=20_000, nq=300, ncomp=8)
    Q = w["queries"]
    ix = bang.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], w["M"])
    q = torch.from_numpy(Q).cuda()
    res = {}
    for src in (0, 1):
        ids = torch.empty((len(Q), 10), dtype=torch.int32, device="cuda")
        dist = torch.empty((len(Q), 10), dtype=torch.float32, device="cuda")
        status = torch.empty(len(Q), dtype=torch.int32, device="cuda")
        ix.search(q, 10, 96, ids, dist, bang.make_params(mode=bang.BANG_MODE_PQ_BF16,
                                                         table_source=src, out_status=status))
        torch.cuda.synchronize()
        assert (status.cpu().numpy() == 0).all()
        res[src] = ids.cpu().numpy().view(np.uint32)
    o = oracle.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], w["M"]).search(Q, 10, 96)
    r_o = oracle.recall_at_k(o["ids"], w["gt_ids"], 10)
    for src in (0, 1):
        assert abs(oracle.recall_at_k(res[src], w["gt_ids"], 10) - r_o) <= 0.005 + 1.0 / (10 * len(Q))
    assert (res[0] == res[1]).mean() > 0.97
    ix.close()


@pytest.mark.parametrize("which", ["u8", "f32", "i8"])
def test_tf32_tables_within_the_tf32_bound(which):
    # both operands rounded to TF32 (10 mantissa bits, relative error 2^-11
    # each), products exact, FP32 accumulation: every entry lies within
    # 2 * 2^-10 * sum_j |q_j| |c_j| of the exact table, plus the FP32 bound of
    # the three-way form; and the rounding is really applied (some entries
    # leave the FP32 bound)
    w = _workload(which)
    Q = w["queries"]
    M, d = w["M"], Q.shape[1]
    T = _tc(w, Q, bf16=False, tf32=True)
    off = oracle.chunk_offsets(d, M)
    cb = w["codebook"].astype(np.float64)
    outside = 0
    for qi in range(0, len(Q), max(1, len(Q) // 25)):
        ref = oracle.adc_table(Q[qi].astype(np.float32), M, w["codebook"]).astype(np.float64)
        qf = Q[qi].astype(np.float64)
        for s in range(M):
            o, ds = off[s], off[s + 1] - off[s]
            C = cb[256 * o: 256 * o + 256 * ds].reshape(256, ds)
            scale = (qf[o:o + ds] ** 2).sum() + (C ** 2).sum(1)
            cross = (np.abs(qf[o:o + ds])[None, :] * np.abs(C)).sum(1)
            err = np.abs(T[qi, s] - ref[s])
            fp32_bound = 4e-6 * scale + 2e-3
            assert (err <= 2.0 ** -9 * cross + fp32_bound).all(), (which, qi, s, err.max())
            outside += int((err > fp32_bound).sum())
    assert outside > 0


def test_fp32_searches_on_tensor_core_tables():
    # the FP32 search mode reading tables from the tensor cores: the
    # three-way (about FP32) tables keep recall within 0.005 of the bit-exact
    # per-warp tables; the TF32 tables are reported against the same bar
    w = cases.clustered(n=20_000, nq=300, ncomp=8)
    Q = w["queries"]
    ix = bang.Index(w["base"], w["codebook"], w["codes"], w["adj"], w["medoid"], w["M"])
    q = torch.from_numpy(Q).cuda()
    rec = {}
    for src in (0, 1, 2):
        ids = torch.empty((len(Q), 10), dtype=torch.int32, device="cuda")
        dist = torch.empty((len(Q), 10), dtype=torch.float32, device="cuda")
        status = torch.empty(len(Q), dtype=torch.int32, device="cuda")
        ix.search(q, 10, 96, ids, dist, bang.make_params(mode=bang.BANG_MODE_PQ_F32, table_source=src,
                                                         out_status=status))
        torch.cuda.synchronize()
        assert (status.cpu().numpy() == 0).all()
        rec[src] = oracle.recall_at_k(ids.cpu().numpy().view(np.uint32), w["gt_ids"], 10)
    assert abs(rec[1] - rec[0]) <= 0.005 + 1.0 / (10 * len(Q))
    assert rec[2] >= rec[0] - 0.1
    ix.close()
