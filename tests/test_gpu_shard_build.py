"""GPU build of the overlapping-shard graph (§2.2) against the oracle's
orc_shard_graph: the adjacency and the shard assignment must be equal byte
for byte (u8, i8 and f32; several shards per point; batches that span many
rounds; a ragged point count; a round large enough that some reverse-edge
lists go to the large-list kernel)."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2401_11324_gb300 as bang  # noqa: E402


def _data(rng, n, d, dtype, ncomp=6):
    if dtype == "f32":
        cen = rng.normal(0, 3, size=(ncomp, d))
        X = (cen[rng.integers(0, ncomp, n)] + rng.normal(size=(n, d))).astype(np.float32)
    elif dtype == "i8":
        cen = rng.integers(-90, 90, size=(ncomp, d))
        X = np.clip(cen[rng.integers(0, ncomp, n)] + rng.normal(0, 12, size=(n, d)), -128, 127)
        X = np.rint(X).astype(np.int8)
    else:
        cen = rng.integers(20, 235, size=(ncomp, d))
        X = np.clip(cen[rng.integers(0, ncomp, n)] + rng.normal(0, 15, size=(n, d)), 0, 255)
        X = np.rint(X).astype(np.uint8)
    return X


CASES = [
    # dtype, n, d, S, ell, R, Lb, alpha, batch_frac, log2z
    ("u8", 3001, 32, 6, 2, 16, 24, 1.2, 0.05, 14),
    ("u8", 4000, 128, 8, 2, 64, 64, 1.2, 0.02, 16),
    ("i8", 2003, 100, 4, 2, 32, 32, 1.2, 0.05, 15),
    ("f32", 1500, 24, 5, 3, 12, 20, 1.2, 0.1, 14),
    ("f32", 700, 130, 3, 1, 8, 16, 1.0, 0.2, 12),
    ("u8", 997, 20, 1, 1, 16, 32, 1.3, 0.05, 13),
    ("u8", 3000, 16, 2, 2, 128, 32, 1.2, 1.0, 14),     # one pass-2 round of every member
    ("u8", 6000, 24, 1, 1, 64, 48, 1.2, 1.0, 15),      # hubs with over 750 reverse candidates
    ("u8", 60000, 128, 16, 2, 64, 64, 1.2, 0.02, 16),  # the large configurations' settings
]


@pytest.mark.parametrize("case", CASES, ids=["%s-n%d-d%d-S%d-l%d-R%d" % c[:6] for c in CASES])
def test_shard_graph_equals_oracle(case):
    dt, n, d, S, ell, R, Lb, alpha, frac, lz = case
    rng = np.random.default_rng(n + d + S)
    X = _data(rng, n, d, dt)
    centres = X[rng.choice(n, S, replace=False)].astype(np.float32)
    want, wsh = oracle.shard_graph(X, centres, ell, R, Lb, alpha, frac, lz)
    got, gsh = bang.bang_build_shard_graph(X, centres, ell, R, Lb, alpha, frac, lz)
    assert (gsh == wsh).all()
    bad = np.argwhere(got != want)
    assert bad.size == 0, (bad[:5], got[bad[0][0]], want[bad[0][0]])


def test_shard_graph_device_buffers():
    rng = np.random.default_rng(5)
    X = _data(rng, 2500, 64, "u8")
    centres = X[rng.choice(2500, 4, replace=False)].astype(np.float32)
    want, _ = oracle.shard_graph(X, centres, 2, 32, 32, 1.2, 0.05, 14)
    Xd = torch.from_numpy(X).cuda()
    adj = torch.zeros((2500, 32), dtype=torch.int32, device="cuda")
    bang.bang_build_shard_graph(Xd, centres, 2, 32, 32, 1.2, 0.05, 14, adj=adj)
    assert (adj.cpu().numpy().view(np.uint32) == want).all()
