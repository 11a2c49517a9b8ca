"""Pins for the CPU oracle: each test checks it against something the paper or
the mathematics fixes (closed forms, published hash vectors, the paper's
worked example, invariants, brute force on tiny inputs), never against a
retyped copy of itself."""
import ctypes
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

NONE = oracle.NONE
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers

def lossless_u8(X):
    """PQ with one dimension per subspace and the codebook C[s][c] = c: the
    codes are the points themselves and ADC equals the exact distance."""
    n, d = X.shape
    cb = np.tile(np.arange(256, dtype=np.float32), d)
    return cb, X.astype(np.uint8).copy()


def complete_graph(n):
    adj = np.full((n, max(n - 1, 1)), NONE, np.uint32)
    for i in range(n):
        adj[i, :n - 1] = [j for j in range(n) if j != i]
    return adj


def brute_ids(X, q, k):
    d = ((X.astype(np.int64) - q.astype(np.int64)) ** 2).sum(1)
    order = np.lexsort((np.arange(len(d)), d))
    return order[:k], d[order[:k]]


# ---------------------------------------------------------------- FNV-1a, Bloom (§4.3, §6.3)

def test_fnv1a_published_vectors():
    # Test vectors published with the FNV hash definition.
    assert oracle.fnv1a32(b"") == 0x811C9DC5
    assert oracle.fnv1a32(b"a") == 0xE40C292C
    assert oracle.fnv1a32(b"foobar") == 0xBF9CF968
    assert oracle.fnv1a64(b"") == 0xCBF29CE484222325
    assert oracle.fnv1a64(b"a") == 0xAF63DC4C8601EC8C
    assert oracle.fnv1a64(b"foobar") == 0x85944171F73967E8


def test_bloom_hashes_little_endian_id_bytes():
    b = oracle.Bloom(20)
    ident = int.from_bytes(b"abcd", "little")
    h64 = oracle.fnv1a64(b"abcd")
    p1, p2 = b.positions(ident)
    assert p1 == oracle.fnv1a32(b"abcd") & ((1 << 20) - 1)
    assert p2 == ((h64 >> 32) ^ (h64 & 0xFFFFFFFF)) & ((1 << 20) - 1)


def test_bloom_no_false_negatives_and_fp_rate():
    rng = np.random.default_rng(7)
    log2z, n_ins, n_test = 14, 2000, 40000
    ids = rng.choice(1 << 30, size=n_ins + n_test, replace=False)
    b = oracle.Bloom(log2z)
    for i in ids[:n_ins]:
        b.insert(int(i))
    assert all(b.test(int(i)) for i in ids[:n_ins])
    fp = sum(b.test(int(i)) for i in ids[n_ins:]) / n_test
    z = 1 << log2z
    expect = (1 - math.exp(-2 * n_ins / z)) ** 2
    sigma = math.sqrt(expect * (1 - expect) / n_test)
    assert abs(fp - expect) < 3 * sigma + 0.15 * expect


# ---------------------------------------------------------------- PQ (§4)

def test_chunk_offsets_uneven_split():
    off = oracle.chunk_offsets(128, 74)
    sizes = np.diff(off)
    assert off[-1] == 128 and len(sizes) == 74
    assert (sizes[:54] == 2).all() and (sizes[54:] == 1).all()
    assert (np.diff(oracle.chunk_offsets(96, 48)) == 2).all()


def test_adc_table_closed_form():
    d, M = 8, 2
    c = np.arange(256, dtype=np.float64)
    cb = np.concatenate([(c[:, None] + 0.25 * np.arange(4)[None, :] + 3 * s).ravel()
                         for s in range(M)]).astype(np.float32)
    q = np.array([0.5, -1.0, 2.0, 7.25, 100.0, 3.5, 0.0, 255.0], np.float32)
    T = oracle.adc_table(q, M, cb)
    for s in range(M):
        for cc in (0, 1, 17, 128, 255):
            exact = sum((Fraction(float(q[4 * s + j])) - Fraction(cc) - Fraction(j, 4) - 3 * s) ** 2
                        for j in range(4))
            assert Fraction(float(T[s, cc])) == exact


def test_adc_dist_is_sum_of_selected_entries():
    rng = np.random.default_rng(1)
    M = 32
    T = rng.integers(0, 2000, size=(M, 256)).astype(np.float32)
    for _ in range(20):
        code = rng.integers(0, 256, size=M).astype(np.uint8)
        assert oracle.adc_dist(T, code) == float(sum(int(T[s, code[s]]) for s in range(M)))


def test_bf16_rounding_closed_form():
    # BF16 keeps 8 significant bits.  Representable values stay; halfway
    # cases go to the neighbour whose last kept bit is 0; anything above the
    # halfway point rounds up (worked by hand from the binary expansions).
    u = 2.0 ** -8                          # half a BF16 step at 1.0 (step 2^-7)
    for x in (1.0, 1.5, 3.0, 255.0, 2.0 ** -10, 0.0, 2.0 ** 20):
        assert oracle.round_bf16(x) == x
    assert oracle.round_bf16(1 + u) == 1.0                        # tie, 1.0 is even
    assert oracle.round_bf16(1 + 3 * u) == 1 + 4 * u              # tie, 1 + 2^-6 is even
    assert oracle.round_bf16(1 + u + 2.0 ** -20) == 1 + 2 * u     # above the tie
    assert oracle.round_bf16(1 + u - 2.0 ** -20) == 1.0           # below the tie
    assert oracle.round_bf16(257.0) == 256.0                      # 8 bits: steps of 2 at 256
    assert oracle.round_bf16(259.0) == 260.0                      # tie, 260 = 0b100000100 even
    assert oracle.round_bf16(65535.0) == 65536.0
    T = np.array([[1 + u, 1 + 3 * u, 257.0, 259.0] + [0.0] * 252], np.float32)
    assert oracle.adc_table_bf16(T)[0, :4].tolist() == [1.0, 1 + 4 * u, 256.0, 260.0]


def test_bf16_search_equals_fp32_when_entries_are_representable():
    # On the chain graph every entry the search reads is (13 - c)^2 <= 169,
    # an integer below 256 and so exact in BF16: the visits equal the FP32
    # table's (entries of far centroids, up to 242^2, do round).
    n = 21
    X = np.arange(n, dtype=np.uint8)[:, None]
    adj = np.full((n, 2), NONE, np.uint32)
    for i in range(n):
        nb = [j for j in (i - 1, i + 1) if 0 <= j < n]
        adj[i, :len(nb)] = nb
    cb, codes = lossless_u8(X)
    ix = oracle.Index(X, cb, codes, adj, 0, 1)
    q = np.array([[13]], np.uint8)
    T = oracle.adc_table(q[0].astype(np.float32), 1, cb)
    assert (oracle.adc_table_bf16(T) != T).any()
    for L in (1, 2, 3, 5):
        a = ix.search(q, k=1, L=L, trace_cap=64)
        b = ix.search(q, k=1, L=L, trace_cap=64, bf16=True)
        assert b["trace"][0].tolist() == a["trace"][0].tolist() and b["ids"][0, 0] == a["ids"][0, 0]


def test_bf16_rounding_changes_the_visit():
    # Query (0, 0), lossless 1-dimension subspaces.  Point 1 = (17, 0) has
    # FP32 distance 289, which BF16 rounds to 288 (a tie between 288 and 290
    # going to the even 288); point 2 = (12, 12) has 144 + 144 = 288 exactly.
    # With L = 1 the FP32 table keeps point 2 (288 < 289) after expanding the
    # far medoid 0; the BF16 table sees a tie and keeps the smaller id, 1.
    # The re-rank returns the nearest expanded node: 2 for FP32, 1 for BF16.
    X = np.array([[200, 200], [17, 0], [12, 12]], np.uint8)
    cb, codes = lossless_u8(X)
    ix = oracle.Index(X, cb, codes, complete_graph(3), 0, 2)
    q = np.zeros((1, 2), np.uint8)
    a = ix.search(q, k=1, L=1, trace_cap=8)
    b = ix.search(q, k=1, L=1, trace_cap=8, bf16=True)
    assert a["trace"][0][:2].tolist() == [0, 2] and a["ids"][0, 0] == 2 and a["dist"][0, 0] == 288.0
    assert b["trace"][0][:2].tolist() == [0, 1] and b["ids"][0, 0] == 1 and b["dist"][0, 0] == 289.0


def test_bf16_mode_worklist_of_all_points_equals_bruteforce():
    rng = np.random.default_rng(23)
    n = 30
    X = rng.integers(0, 256, size=(n, 16)).astype(np.uint8)
    cb = rng.normal(128, 40, size=256 * 16).astype(np.float32)
    codes = rng.integers(0, 256, size=(n, 4)).astype(np.uint8)
    ix = oracle.Index(X, cb, codes, complete_graph(n), 3, 4)
    Q = rng.integers(0, 256, size=(6, 16)).astype(np.uint8)
    r = ix.search(Q, k=5, L=n, log2z=18, bf16=True)
    for qi in range(len(Q)):
        ids, dd = brute_ids(X, Q[qi], 5)
        assert r["ids"][qi].tolist() == ids.tolist()
        assert r["dist"][qi].tolist() == dd.astype(np.float32).tolist()


def test_q8_table_closed_form():
    # Subspace 0: entries 2*pi(c), pi a permutation of 0..255 (width 510);
    # subspace 1: 100 + c (width 255); subspace 2: constant (width 0).  The
    # widest subspace fixes the scale 255/510 = 1/2 exactly, so subspace 0
    # maps to pi(c), subspace 1 to c/2 rounded half to even, subspace 2 to 0.
    perm = (np.arange(256) * 37) % 256
    T = np.stack([2.0 * perm, 100.0 + np.arange(256), np.full(256, 7.0)]).astype(np.float32)
    Q = oracle.adc_table_q8(T)
    assert Q[0].tolist() == perm.tolist()
    assert Q[1].tolist() == [round(c / 2) for c in range(256)]     # Python rounds halves to even
    assert Q[1][1] == 0 and Q[1][3] == 2 and Q[1][5] == 2 and Q[1][255] == 128
    assert not Q[2].any()
    # the distance is the integer sum of the selected entries
    assert oracle.adc_dist_q8(Q, np.array([5, 7, 9], np.uint8)) == 185 + 4 + 0


def test_q8_table_invariants():
    rng = np.random.default_rng(21)
    for trial in range(20):
        M = int(rng.integers(1, 40))
        T = (rng.gamma(2.0, 1.0, size=(M, 256)) * rng.uniform(0.1, 1e4, size=(M, 1))).astype(np.float32)
        Q = oracle.adc_table_q8(T).astype(np.int64)
        lo = T.astype(np.float64).min(1)
        width = T.astype(np.float64).max(1) - lo
        g = width.max()
        assert (Q.min(1) == 0).all()                       # every subspace's minimum maps to 0
        assert Q[int(np.argmax(width))].max() == 255       # the widest subspace spans the range
        assert Q.max() <= 255
        err = np.abs(Q * g / 255.0 - (T - lo[:, None]))
        assert (err <= g / 510.0 * (1 + 1e-5) + 1e-6 * T.max()).all()
        for s in range(M):                                 # order within a subspace is kept
            o = np.argsort(T[s], kind="stable")
            assert (np.diff(Q[s][o]) >= 0).all()
    assert not oracle.adc_table_q8(np.full((4, 256), 3.5, np.float32)).any()


def test_adc_dist_summation_tree():
    # Reading of §4.4 (order of the segment sums): 8 strided partials, then
    # butterfly p_r += p_(r^4), p_r += p_(r^2), p_r += p_(r^1).  Values
    # chosen so that any other order of the additions rounds differently.
    M = 16
    T = np.zeros((M, 256), np.float32)
    vals = [1.0, 2.0 ** -24, 2.0 ** -24, 0.0, 0.0, 0.0, 0.0, 0.0,
            2.0 ** -24, 2.0 ** -24, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0]
    for s, v in enumerate(vals):
        T[s, 0] = v
    code = np.zeros(M, np.uint8)
    f = np.float32
    p = [f(0)] * 8
    for s in range(M):
        p[s & 7] = f(p[s & 7] + f(vals[s]))
    for h in (4, 2, 1):
        p = [f(p[r] + p[r ^ h]) for r in range(8)]
    got = oracle.adc_dist(T, code)
    assert got == float(p[0])
    seq = f(0)
    for v in vals:
        seq = f(seq + f(v))
    assert got != float(seq)          # plain left-to-right order would differ


def test_pq_encode_closed_form_and_ties():
    d, M = 8, 2
    rng = np.random.default_rng(2)
    cb = rng.integers(0, 200, size=256 * d).astype(np.float32)
    cb[256 * 4 + 9 * 4: 256 * 4 + 10 * 4] = cb[256 * 4 + 3 * 4: 256 * 4 + 4 * 4]  # s=1: c9 == c3
    X = np.zeros((3, d), np.float32)
    X[0, :4] = cb[5 * 4:6 * 4]; X[0, 4:] = cb[256 * 4 + 200 * 4: 256 * 4 + 201 * 4]
    X[1, :4] = cb[0:4]; X[1, 4:] = cb[256 * 4 + 9 * 4: 256 * 4 + 10 * 4]
    X[2, :4] = cb[255 * 4:256 * 4]; X[2, 4:] = cb[256 * 4 + 255 * 4: 256 * 4 + 256 * 4]
    codes = oracle.pq_encode(X, M, cb)
    assert codes[0].tolist() == [5, 200]
    assert codes[1].tolist() == [0, 3]          # tie between c3 and c9 -> smaller id
    assert codes[2].tolist() == [255, 255]


def test_kmeans_fixed_point_and_separated_clusters():
    rng = np.random.default_rng(3)
    d, M = 8, 2
    # 256 distinct points, initialised at themselves: a fixed point, objective 0.
    P = rng.permutation(256 * 256)[:256]
    X = np.stack([(P // 256) % 256, P % 256, P % 7, P % 5, P % 11, P % 13, P % 3, P % 17], 1)
    X = X.astype(np.float32)
    _, uniq = np.unique(X[:, :4], axis=0, return_index=True)
    _, uniq2 = np.unique(X[:, 4:], axis=0, return_index=True)
    assert len(uniq) == 256
    init = np.stack([np.arange(256), np.arange(256)])
    cb, tr = oracle.pq_train(X, M, np.arange(256), init, 3, return_trace=True)
    assert np.array_equal(cb[:256 * 4].reshape(256, 4), X[:, :4])
    assert tr[0].tolist() == [0.0, 0.0, 0.0]
    # 256 tight, well separated clusters of 6 points: after one Lloyd step
    # every centroid is its cluster mean.
    centres = rng.permutation(256 * 256)[:256]
    C = np.stack([centres // 256, centres % 256, (centres * 7) % 251, (centres * 3) % 241], 1)
    C = (C * 100.0).astype(np.float64)
    off = rng.normal(0, 1.0, size=(256, 6, 4))
    Y = (C[:, None, :] + off).reshape(-1, 4)
    Y = np.concatenate([Y, Y], 1).astype(np.float32)
    init = np.stack([np.arange(256) * 6, np.arange(256) * 6])
    cb, tr = oracle.pq_train(Y, M, np.arange(len(Y)), init, 2, return_trace=True)
    means = Y[:, :4].astype(np.float64).reshape(256, 6, 4).mean(1)
    assert np.allclose(cb[:256 * 4].reshape(256, 4), means, rtol=0, atol=1e-3)
    assert tr[0, 1] <= tr[0, 0]


def test_kmeans_objective_non_increasing():
    rng = np.random.default_rng(4)
    X = rng.normal(size=(3000, 16)).astype(np.float32)
    init = np.stack([rng.choice(3000, 256, replace=False) for _ in range(4)])
    _, tr = oracle.pq_train(X, 4, np.arange(3000), init, 8, return_trace=True)
    assert (np.diff(tr, axis=1) <= 1e-9 * tr[:, :-1]).all()


def test_medoid_closed_form():
    X = np.zeros((7, 3), np.float32)
    X[:, 0] = [0, 1, 2, 10, 11, 12, 6]      # mean 6 -> point 6
    assert oracle.medoid(X) == 6
    Y = np.array([[0], [2], [4], [6]], np.uint8)   # mean 3: points 1 and 2 tie -> 1
    assert oracle.medoid(Y) == 1


# ---------------------------------------------------------------- exact distance (§4.8)

def test_exact_dist_integer_types_exact():
    rng = np.random.default_rng(5)
    for dt, lo, hi in ((np.uint8, 0, 256), (np.int8, -128, 128)):
        a = rng.integers(lo, hi, size=100).astype(dt)
        b = rng.integers(lo, hi, size=100).astype(dt)
        assert oracle.exact_dist(a, b) == float(((a.astype(np.int64) - b.astype(np.int64)) ** 2).sum())
    a = np.full(128, 255, np.uint8)
    b = np.zeros(128, np.uint8)
    assert oracle.exact_dist(a, b) == 128 * 255 ** 2


def test_exact_dist_f32_error_bound_and_order():
    rng = np.random.default_rng(6)
    for d in (96, 100, 128, 200):
        a = rng.normal(size=d).astype(np.float32)
        b = rng.normal(size=d).astype(np.float32)
        ref = float(((a.astype(np.float64) - b.astype(np.float64)) ** 2).sum())
        got = oracle.exact_dist(a, b)
        assert abs(got - ref) <= (d + 2) * 2.0 ** -24 * ref
    # Strided-partials tree (the order is a reading: the paper does not fix
    # it).  Squared differences of 2^-24 are exact, so the only rounding is in
    # the additions.  Case 1: dims 0..3 share partial 0, so three 2^-24 terms
    # each vanish against 1.0 -> exactly 1.0 (a tree splitting them would
    # give 1 + 2^-23).  Case 2: dims 4..6 share partial 1 (sum 3*2^-24), which
    # meets 1.0 once -> 1 + 2^-22 by round-to-even (left-to-right gives 1.0).
    b = np.zeros(8, np.float32)
    a = np.zeros(8, np.float32)
    a[0] = 1.0
    a[1:4] = 2.0 ** -12
    assert oracle.exact_dist(a, b) == 1.0
    a = np.zeros(8, np.float32)
    a[0] = 1.0
    a[4:7] = 2.0 ** -12
    assert oracle.exact_dist(a, b) == 1.0 + 2.0 ** -22


# ---------------------------------------------------------------- the paper's worked example

def _read_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "toy_workflow.txt"))
            if l.strip() and not l.startswith("#")]
    g = {"b": {}, "d": []}
    for r in rows:
        if r[0] == "query":
            g["q"] = (int(r[1]), int(r[2]))
        elif r[0] == "table_b":
            g["b"][int(r[1])] = int(r[3])
        elif r[0] == "table_d":
            g["d"].append((int(r[2]), int(r[3])))
        elif r[0] == "sorted_candidates":
            g["sorted"] = [int(x) for x in r[1:]]
        elif r[0] == "top2":
            g["top2"] = [int(x) for x in r[1:]]
    return g


def _point_at(q, dist):
    """A 3-D integer point at the given squared distance from (q, 0)."""
    for a in range(0, 90):
        for b in range(0, a + 1):
            for c in range(0, 8):
                if a * a + b * b + c * c == dist:
                    return (q[0] + a, q[1] + b, c)
    raise AssertionError(dist)


def test_worked_example_rerank():
    g = _read_golden()
    q = g["q"]
    cand = [n for n, _ in g["d"]]
    dist_d = dict(g["d"])
    X = np.zeros((12, 3), np.uint8)
    for node in range(12):
        X[node] = _point_at(q, dist_d.get(node, g["b"][node]))
    qv = np.array([q[0], q[1], 0], np.uint8)
    for node, dd in g["d"]:
        assert oracle.exact_dist(qv, X[node]) == dd
    # The figure's graph is lost: search the subgraph of the eight candidates
    # (complete among them) from the first candidate, with a worklist large
    # enough to visit all of them, then re-rank.
    adj = np.full((12, 7), NONE, np.uint32)
    for i in cand:
        adj[i] = [j for j in cand if j != i]
    cb, codes = lossless_u8(X)
    ix = oracle.Index(X, cb, codes, adj, cand[0], 3)
    r = ix.search(qv[None], k=8, L=8, log2z=16, trace_cap=16)
    assert sorted(r["trace"][0][:r["iters"][0]].tolist()) == sorted(cand)
    assert r["ids"][0].tolist() == g["sorted"]
    r2 = ix.search(qv[None], k=2, L=8, log2z=16)
    assert r2["ids"][0].tolist() == g["top2"]


# ---------------------------------------------------------------- search (Alg. 1 / Alg. 2)

def test_lossless_pq_equals_exact_distance():
    rng = np.random.default_rng(8)
    X = rng.integers(0, 256, size=(50, 128)).astype(np.uint8)
    cb, codes = lossless_u8(X)
    q = rng.integers(0, 256, size=128).astype(np.uint8)
    T = oracle.adc_table(q.astype(np.float32), 128, cb)
    for i in range(50):
        assert oracle.adc_dist(T, codes[i]) == oracle.exact_dist(q, X[i])


def test_chain_graph_visit_order():
    # Points 0..20 on a line, chain graph i <-> i+1, entry 0, query 13.
    # Worked by hand from Alg. 1 with the seen-set filter of Alg. 2:
    # L=1 and L=2 expand 0..13 (14 is seen at 13 but never beats it);
    # L=3 also expands 14, whose new neighbour 15 falls off the list.
    n = 21
    X = np.arange(n, dtype=np.uint8)[:, None]
    adj = np.full((n, 2), NONE, np.uint32)
    for i in range(n):
        nb = [j for j in (i - 1, i + 1) if 0 <= j < n]
        adj[i, :len(nb)] = nb
    cb, codes = lossless_u8(X)
    ix = oracle.Index(X, cb, codes, adj, 0, 1)
    q = np.array([[13]], np.uint8)
    for L, last in ((1, 13), (2, 13), (3, 14)):
        r = ix.search(q, k=1, L=L, log2z=16, trace_cap=64)
        it = int(r["iters"][0])
        assert r["trace"][0][:it].tolist() == list(range(last + 1))
        assert r["ids"][0, 0] == 13 and r["dist"][0, 0] == 0.0
    r = ix.search(q, k=3, L=3, log2z=16)
    assert r["ids"][0].tolist() == [13, 12, 14]      # (distance, id) ties: 12 before 14


def test_q8_chain_graph_visit_order():
    # The chain graph of test_chain_graph_visit_order on the 8-bit table.
    # With the lossless codebook and query 13 the FP32 entries are (13-c)^2,
    # widest 242^2 = 58564, so the scale is 255/58564 and points 0, 1, 2
    # (169, 144, 121) quantise to 1 while 3..20 (at most 100) quantise to 0.
    # Worked by hand: L=1 stops after 0 (1 ties with 0 and loses on id);
    # L=2 stops after 0, 1; L=3 expands 0..5: 3 enters at distance 0 and
    # every later point ties at 0 and falls off behind smaller ids once 6
    # arrives.  The re-rank then returns the nearest expanded node.
    n = 21
    X = np.arange(n, dtype=np.uint8)[:, None]
    adj = np.full((n, 2), NONE, np.uint32)
    for i in range(n):
        nb = [j for j in (i - 1, i + 1) if 0 <= j < n]
        adj[i, :len(nb)] = nb
    cb, codes = lossless_u8(X)
    ix = oracle.Index(X, cb, codes, adj, 0, 1)
    q = np.array([[13]], np.uint8)
    Q = oracle.adc_table_q8(oracle.adc_table(q[0].astype(np.float32), 1, cb))
    assert Q[0][:21].tolist() == [1, 1, 1] + [0] * 18
    for L, trace, best in ((1, [0], 0), (2, [0, 1], 1), (3, [0, 1, 2, 3, 4, 5], 5)):
        r = ix.search(q, k=1, L=L, log2z=16, trace_cap=64, q8=True)
        it = int(r["iters"][0])
        assert r["trace"][0][:it].tolist() == trace
        assert r["ids"][0, 0] == best and r["dist"][0, 0] == float((13 - best) ** 2)


def test_q8_mode_worklist_of_all_points_equals_bruteforce():
    # With L >= n on a complete graph every point is expanded, so the re-rank
    # returns the exact k-NN whatever the table's precision.
    rng = np.random.default_rng(22)
    n = 30
    X = rng.integers(0, 256, size=(n, 16)).astype(np.uint8)
    cb = rng.normal(128, 40, size=256 * 16).astype(np.float32)
    codes = rng.integers(0, 256, size=(n, 4)).astype(np.uint8)
    ix = oracle.Index(X, cb, codes, complete_graph(n), 3, 4)
    Q = rng.integers(0, 256, size=(6, 16)).astype(np.uint8)
    r = ix.search(Q, k=5, L=n, log2z=18, q8=True)
    for qi in range(len(Q)):
        ids, dd = brute_ids(X, Q[qi], 5)
        assert r["ids"][qi].tolist() == ids.tolist()
        assert r["dist"][qi].tolist() == dd.astype(np.float32).tolist()
        assert r["iters"][qi] == n


def test_complete_graph_equals_bruteforce():
    rng = np.random.default_rng(9)
    for trial in range(5):
        n = int(rng.integers(8, 40))
        X = rng.integers(0, 256, size=(n, 16)).astype(np.uint8)
        cb, codes = lossless_u8(X)
        med = int(rng.integers(0, n))
        ix = oracle.Index(X, cb, codes, complete_graph(n), med, 16)
        Q = rng.integers(0, 256, size=(6, 16)).astype(np.uint8)
        for L in (3, 5, 8):
            k = 3
            r = ix.search(Q, k=k, L=L, log2z=18)
            for qi in range(len(Q)):
                ids, dd = brute_ids(X, Q[qi], k)
                assert r["ids"][qi].tolist() == ids.tolist()
                assert r["dist"][qi].tolist() == dd.astype(np.float32).tolist()
                topL, _ = brute_ids(X, Q[qi], L)
                assert r["iters"][qi] == (L if med in topL.tolist() else L + 1)


def test_exact_mode_complete_graph_equals_bruteforce():
    # Exact-distance variant (§5.2): exact distances in the loop, no re-rank;
    # on a complete graph the worklist after the first expansion holds the L
    # nearest points, so its first k are the exact k-NN.
    rng = np.random.default_rng(16)
    n = 40
    X = rng.normal(size=(n, 12)).astype(np.float32)
    cb = rng.normal(size=256 * 12).astype(np.float32)          # unused by the exact mode
    codes = rng.integers(0, 256, size=(n, 3)).astype(np.uint8)
    ix = oracle.Index(X, cb, codes, complete_graph(n), 7, 3)
    Q = rng.normal(size=(5, 12)).astype(np.float32)
    r = ix.search(Q, k=4, L=6, log2z=18, exact=True)
    ref = ((X[None].astype(np.float64) - Q[:, None].astype(np.float64)) ** 2).sum(-1)
    for qi in range(5):
        assert r["ids"][qi].tolist() == np.argsort(ref[qi])[:4].tolist()
        for j, i in enumerate(r["ids"][qi]):
            assert abs(r["dist"][qi][j] - ref[qi][i]) <= 1e-5 * ref[qi][i]
        top6 = np.argsort(ref[qi])[:6].tolist()
        assert r["iters"][qi] == (6 if 7 in top6 else 7)


def test_full_worklist_visits_every_reachable_node():
    # With L >= n on a connected graph and a filter without false positives
    # in practice (z = 2^22 bits for <= 64 ids), every node is expanded and
    # the re-rank is exact k-NN.
    rng = np.random.default_rng(10)
    for trial in range(5):
        n = 64
        X = rng.integers(0, 256, size=(n, 8)).astype(np.uint8)
        R = 4
        adj = np.full((n, R), NONE, np.uint32)
        perm = rng.permutation(n)
        for t in range(n):                         # a cycle keeps it connected
            adj[perm[t], 0] = perm[(t + 1) % n]
        for i in range(n):
            extra = [j for j in rng.choice(n, size=6, replace=False) if j != i and j != adj[i, 0]]
            adj[i, 1:1 + min(3, len(extra))] = extra[:3]
        cb, codes = lossless_u8(X)
        ix = oracle.Index(X, cb, codes, adj, int(perm[0]), 8)
        Q = rng.integers(0, 256, size=(4, 8)).astype(np.uint8)
        r = ix.search(Q, k=10, L=n, log2z=22)
        for qi in range(len(Q)):
            ids, _ = brute_ids(X, Q[qi], 10)
            assert r["ids"][qi].tolist() == ids.tolist()
            assert r["iters"][qi] == n


def test_padding_when_fewer_than_k_reachable():
    X = np.array([[0], [5], [9], [200]], np.uint8)
    adj = np.array([[1], [0], [NONE], [NONE]], np.uint32)
    cb, codes = lossless_u8(X)
    ix = oracle.Index(X, cb, codes, adj, 0, 1)
    r = ix.search(np.array([[4]], np.uint8), k=4, L=4, log2z=16)
    assert r["ids"][0].tolist() == [1, 0, NONE, NONE]
    assert r["dist"][0, 0] == 1.0 and r["dist"][0, 1] == 16.0 and np.isinf(r["dist"][0, 2:]).all()


def test_iteration_cap_status():
    n = 30
    X = np.arange(n, dtype=np.uint8)[:, None] * 3
    adj = np.full((n, 2), NONE, np.uint32)
    for i in range(n):
        nb = [j for j in (i - 1, i + 1) if 0 <= j < n]
        adj[i, :len(nb)] = nb
    cb, codes = lossless_u8(X)
    ix = oracle.Index(X, cb, codes, adj, 0, 1)
    r = ix.search(np.array([[87]], np.uint8), k=1, L=2, log2z=16, iter_cap=5)
    assert r["status"][0] == 1 and r["iters"][0] == 5
    r = ix.search(np.array([[87]], np.uint8), k=1, L=2, log2z=16)
    assert r["status"][0] == 0 and r["ids"][0, 0] == 29


def test_rerank_uses_exact_distances():
    # Lossy PQ: the re-rank (§4.8) must order by, and return, exact distances.
    rng = np.random.default_rng(15)
    n, d, M = 400, 16, 4
    X = rng.integers(0, 256, size=(n, d)).astype(np.uint8)
    cb = rng.integers(0, 256, size=256 * d).astype(np.float32)
    codes = oracle.pq_encode(X, M, cb)
    adj = np.stack([rng.choice(np.delete(np.arange(n), i), 10, replace=False) for i in range(n)])
    ix = oracle.Index(X, cb, codes, adj.astype(np.uint32), 0, M)
    Q = rng.integers(0, 256, size=(10, d)).astype(np.uint8)
    r = ix.search(Q, k=8, L=16, log2z=18)
    for qi in range(10):
        ex = ((X[r["ids"][qi]].astype(np.int64) - Q[qi].astype(np.int64)) ** 2).sum(1)
        assert r["dist"][qi].tolist() == ex.astype(np.float32).tolist()
        assert all((ex[i], r["ids"][qi][i]) < (ex[i + 1], r["ids"][qi][i + 1]) for i in range(7))


def test_rerank_of_the_final_worklist_hand_worked():
    # Points 3i on a line, chain graph, query 87, L = 2, five expansions
    # allowed.  By hand: expanding 0, 1, 2, 3, 4 moves the worklist to
    # [5 (not expanded), 4], and the cap stops the search there.  Re-ranking
    # the expanded nodes {0..4} gives 4, 3; re-ranking the final worklist
    # {5, 4} gives 5 (72^2 = 5184), 4 (75^2 = 5625).
    n = 30
    X = np.arange(n, dtype=np.uint8)[:, None] * 3
    adj = np.full((n, 2), NONE, np.uint32)
    for i in range(n):
        nb = [j for j in (i - 1, i + 1) if 0 <= j < n]
        adj[i, :len(nb)] = nb
    cb, codes = lossless_u8(X)
    ix = oracle.Index(X, cb, codes, adj, 0, 1)
    q = np.array([[87]], np.uint8)
    r = ix.search(q, k=2, L=2, log2z=16, iter_cap=5, trace_cap=8)
    assert r["trace"][0][:5].tolist() == [0, 1, 2, 3, 4] and r["status"][0] == 1
    assert r["ids"][0].tolist() == [4, 3] and r["dist"][0].tolist() == [5625.0, 6084.0]
    r = ix.search(q, k=2, L=2, log2z=16, iter_cap=5, rerank_list=True)
    assert r["ids"][0].tolist() == [5, 4] and r["dist"][0].tolist() == [5184.0, 5625.0]


def test_rerank_of_the_final_worklist_equals_the_exact_variant_on_lossless_codes():
    # With lossless codes the PQ distance is the exact distance, so the PQ
    # search and the Exact-distance variant (§5.2) visit the same nodes and
    # end with the same worklist, whose first k entries that variant returns:
    # re-ranking the final worklist must return exactly those, also when the
    # cap leaves entries unexpanded
    rng = np.random.default_rng(31)
    n, d = 300, 6
    X = rng.integers(0, 256, size=(n, d)).astype(np.uint8)
    cb, codes = lossless_u8(X)
    adj = np.stack([rng.choice(np.delete(np.arange(n), i), 8, replace=False)
                    for i in range(n)]).astype(np.uint32)
    ix = oracle.Index(X, cb, codes, adj, 0, d)
    Q = rng.integers(0, 256, size=(12, d)).astype(np.uint8)
    for cap in (None, 6):
        lst = ix.search(Q, k=5, L=20, log2z=18, iter_cap=cap, rerank_list=True)
        ex = ix.search(Q, k=5, L=20, log2z=18, iter_cap=cap, exact=True)
        assert (lst["ids"] == ex["ids"]).all() and (lst["dist"] == ex["dist"]).all()
        assert (lst["iters"] == ex["iters"]).all()


def test_rerank_of_the_final_worklist_returns_exact_distances():
    # lossy PQ: the final worklist is ordered by PQ distance, its re-rank by
    # exact distance, which it also returns; with L >= n on a complete graph
    # the final worklist holds every point, so the result is the brute force
    rng = np.random.default_rng(32)
    n, d, M = 60, 16, 4
    X = rng.integers(0, 256, size=(n, d)).astype(np.uint8)
    cb = rng.integers(0, 256, size=256 * d).astype(np.float32)
    codes = oracle.pq_encode(X, M, cb)
    ix = oracle.Index(X, cb, codes, complete_graph(n), 0, M)
    Q = rng.integers(0, 256, size=(6, d)).astype(np.uint8)
    r = ix.search(Q, k=10, L=n, log2z=18, rerank_list=True)
    for qi in range(6):
        ids, dd = brute_ids(X, Q[qi], 10)
        assert r["ids"][qi].tolist() == ids.tolist()
        assert r["dist"][qi].tolist() == dd.astype(np.float32).tolist()


def test_rejects_L_below_k():
    X = np.zeros((4, 1), np.uint8)
    cb, codes = lossless_u8(X)
    ix = oracle.Index(X, cb, codes, complete_graph(4), 0, 1)
    with pytest.raises(ValueError):
        ix.search(X[:1], k=3, L=2)


def test_iterations_at_least_worklist_size():
    # Every entry of the final worklist has been expanded (§7.7: I >= t).
    rng = np.random.default_rng(11)
    n = 300
    X = rng.integers(0, 256, size=(n, 16)).astype(np.uint8)
    adj = np.stack([rng.choice(np.delete(np.arange(n), i), 12, replace=False) for i in range(n)])
    cb, codes = lossless_u8(X)
    ix = oracle.Index(X, cb, codes, adj.astype(np.uint32), 0, 16)
    r = ix.search(rng.integers(0, 256, size=(20, 16)).astype(np.uint8), k=5, L=24, log2z=18)
    assert (r["iters"] >= 24).all()


# ---------------------------------------------------------------- brute force

def test_bruteforce_matches_lexsort_with_ties():
    rng = np.random.default_rng(12)
    X = rng.integers(0, 4, size=(500, 4)).astype(np.uint8)       # many ties
    Q = rng.integers(0, 4, size=(10, 4)).astype(np.uint8)
    ids, dd = oracle.bruteforce_knn(X, Q, 20)
    for qi in range(10):
        e_ids, e_d = brute_ids(X, Q[qi], 20)
        assert ids[qi].tolist() == e_ids.tolist()
        assert dd[qi].tolist() == e_d.astype(float).tolist()
    Xf = rng.normal(size=(300, 12)).astype(np.float32)
    Qf = rng.normal(size=(5, 12)).astype(np.float32)
    ids, dd = oracle.bruteforce_knn(Xf, Qf, 7)
    ref = ((Xf[None].astype(np.float64) - Qf[:, None].astype(np.float64)) ** 2).sum(-1)
    assert (ids == np.argsort(ref, 1)[:, :7]).all()


# ---------------------------------------------------------------- Vamana (invariants only)

def test_robust_prune_rule():
    rng = np.random.default_rng(13)
    X = rng.normal(size=(200, 8)).astype(np.float32)
    p = 0
    cand = rng.choice(np.arange(1, 200), 80, replace=False)
    alpha, R = 1.2, 12
    out = oracle.robust_prune(X, p, cand, alpha, R)
    d = lambda a, b: float(((X[a].astype(np.float64) - X[b]) ** 2).sum())
    order = sorted(cand.tolist(), key=lambda c: (d(p, c), c))
    assert out[0] == order[0] and len(out) <= R
    kept = out.tolist()
    # kept in increasing distance; none is dominated by an earlier kept one
    for i, a in enumerate(kept):
        for b in kept[:i]:
            assert not (alpha ** 2 * d(b, a) <= d(p, a))
    # when fewer than R are kept, each dropped candidate is dominated by a
    # kept one that precedes it
    if len(kept) < R:
        for c in order:
            if c in kept:
                continue
            assert any(alpha ** 2 * d(b, c) <= d(p, c) for b in kept if (d(p, b), b) < (d(p, c), c))


# ---------------------------------------------------------------- clustered graph construction

def test_cluster_graph_line_alpha1_is_chain():
    # Points on a line (d = 1), one cluster, alpha = 1: the nearest candidate
    # removes every candidate beyond it on its side, so each point keeps its
    # nearest neighbour on either side, the nearer first (ties: smaller id).
    rng = np.random.default_rng(31)
    n = 40
    pos = np.cumsum(rng.integers(1, 4, size=n))             # distinct, gaps 1..3
    assert pos.max() < 256
    ids_by_pos = rng.permutation(n)                         # id of the i-th point from the left
    X = np.zeros((n, 1), np.uint8)
    X[ids_by_pos, 0] = pos
    adj = oracle.cluster_graph(X, np.arange(n), [0, n], [0], R=6, alpha=1.0)
    for i in range(n):
        a = ids_by_pos[i]
        nb = [(int(pos[j] - pos[i]) ** 2, int(ids_by_pos[j])) for j in (i - 1, i + 1) if 0 <= j < n]
        want = [b for _, b in sorted(nb)]
        assert adj[a].tolist() == want + [NONE] * (6 - len(want)), (i, adj[a], want)


def test_cluster_graph_huge_alpha_gives_nearest_lists_and_links():
    # alpha = 1e4 removes nothing (distinct points), so every in-cluster list
    # is the exact R - nx nearest members, except where step 4 gave a point
    # nobody linked to a place at the end of a neighbour's full list.  Rows end
    # with the medoids of the listed clusters, own cluster skipped.
    rng = np.random.default_rng(32)
    ng, per, d, R, nx, nh = 3, 30, 4, 10, 2, 2
    n = ng * per
    X = np.unique(rng.integers(0, 256, size=(n + 20, d)), axis=0)[:n].astype(np.uint8)
    X = X[rng.permutation(n)]
    lab = np.repeat(np.arange(ng), per)[rng.permutation(n)]
    members = np.argsort(lab, kind="stable").astype(np.uint32)
    gstart = np.concatenate([[0], np.cumsum(np.bincount(lab, minlength=ng))])
    medoids = np.array([members[gstart[g]] for g in range(ng)], np.uint32)
    xclu = rng.integers(0, ng, size=(n, nx))
    hclu = np.array([[(g + 1) % ng, (g + 2) % ng] for g in range(ng)])
    adj = oracle.cluster_graph(X, members, gstart, medoids, R, 1e4, nx, xclu, nh, hclu)
    Rin = R - nx
    for g in range(ng):
        P = members[gstart[g]:gstart[g + 1]]
        D = ((X[P].astype(np.int64)[:, None] - X[P].astype(np.int64)[None]) ** 2).sum(-1)
        knn = []
        for a in range(len(P)):
            o = [b for b in np.lexsort((np.arange(len(P)), D[a])) if b != a][:Rin]
            knn.append(o)
        indeg = np.zeros(len(P), int)
        for o in knn:
            indeg[o] += 1
        orphans = set(P[np.where(indeg == 0)[0]].tolist())
        for a in range(len(P)):
            row = adj[P[a]]
            is_med = P[a] == medoids[g]
            keep = min(Rin, R - nh) if is_med else Rin
            exp = [P[b] for b in knn[a]][:keep]
            assert row[:keep - 1].tolist() == exp[:keep - 1]
            assert row[keep - 1] == exp[keep - 1] or int(row[keep - 1]) in orphans
            links = [int(medoids[c]) for c in (hclu[g] if is_med else xclu[P[a]]) if c != g]
            tail = []
            for x in links:
                if x not in tail and x not in row[:keep].tolist():
                    tail.append(x)
            assert row[keep:keep + len(tail)].tolist() == tail
            assert (row[keep + len(tail):] == NONE).all()


def test_cluster_graph_repair_links_an_outlier():
    # A tight group plus one far point: no member keeps the far point (alpha
    # huge: lists are the exact nearest), so step 4 puts it at the end of its
    # nearest neighbour's full list, in place of an entry that keeps another
    # in-link.
    rng = np.random.default_rng(34)
    m, R = 25, 6
    X = np.unique(rng.integers(100, 140, size=(m + 10, 3)), axis=0)[:m - 1].astype(np.uint8)
    X = np.vstack([X, np.array([[250, 250, 250]], np.uint8)])     # outlier = id m-1
    adj = oracle.cluster_graph(X, np.arange(m), [0, m], [0], R=R, alpha=1e4)
    D = ((X.astype(np.int64)[:, None] - X.astype(np.int64)[None]) ** 2).sum(-1)
    knn = [[b for b in np.lexsort((np.arange(m), D[a])) if b != a][:R] for a in range(m)]
    assert all(m - 1 not in knn[a] for a in range(m - 1))
    j = knn[m - 1][0]
    indeg = np.bincount(np.concatenate(knn), minlength=m)
    assert indeg[knn[j][-1]] > 1
    assert adj[j].tolist() == knn[j][:-1] + [m - 1]
    assert adj[m - 1].tolist() == knn[m - 1]


def test_cluster_graph_matches_independent_generator_build():
    # the workload generator builds the same construction with its own code
    # (quickselect, OpenMP over clusters); both must agree bit for bit,
    # including alpha = 1 on small-range integers, where distance ties decide
    import workload
    rng = np.random.default_rng(33)
    for dt, alpha, hi in (("u8", 1.0, 6), ("u8", 1.2, 256), ("i8", 1.2, 128), ("f32", 1.2, 0)):
        ng, n, d, R, nx, nh = 4, 400, 8, 12, 2, 3
        if dt == "f32":
            X = rng.normal(size=(n, d)).astype(np.float32)
        elif dt == "i8":
            X = rng.integers(-hi, hi, size=(n, d)).astype(np.int8)
        else:
            X = rng.integers(0, hi, size=(n, d)).astype(np.uint8)
        lab = rng.integers(0, ng, size=n)
        members = np.argsort(lab, kind="stable").astype(np.uint32)
        gstart = np.concatenate([[0], np.cumsum(np.bincount(lab, minlength=ng))]).astype(np.uint64)
        medoids = np.array([members[gstart[g]] for g in range(ng)], np.uint32)
        xclu = rng.integers(0, ng, size=(n, nx)).astype(np.uint32)
        hclu = rng.integers(0, ng, size=(ng, nh)).astype(np.uint32)
        ref = oracle.cluster_graph(X, members, gstart, medoids, R, alpha, nx, xclu, nh, hclu)
        gen = np.zeros((n, R), np.uint32)
        rc = workload.lib().wl_cluster_graph(
            workload._p(X), {"u8": 0, "i8": 1, "f32": 2}[dt], d, n, workload._p(members),
            workload._p(gstart), ng, workload._p(medoids), R, ctypes.c_float(alpha), nx,
            workload._p(xclu), nh, workload._p(hclu), workload._p(gen))
        assert rc == 0
        assert (gen == ref).all(), (dt, alpha, np.argwhere(gen != ref)[:5])


def test_vamana_invariants():
    rng = np.random.default_rng(14)
    n, d, R = 600, 16, 12
    cen = rng.normal(0, 2, size=(6, d))
    X = (cen[rng.integers(0, 6, n)] + rng.normal(size=(n, d))).astype(np.float32)
    init = np.stack([rng.choice(np.delete(np.arange(n), i), R, replace=False) for i in range(n)])
    med = oracle.medoid(X)
    adj = oracle.vamana_build(X, R, 32, 1.2, med, init.astype(np.uint32),
                              rng.permutation(n).astype(np.uint32))
    for i in range(n):
        row = adj[i]
        ids = row[row != NONE]
        assert len(ids) >= 1 and (row[len(ids):] == NONE).all()
        assert i not in ids.tolist() and len(set(ids.tolist())) == len(ids)
    seen = {med}
    frontier = [med]
    while frontier:
        nxt = []
        for u in frontier:
            for v in adj[u]:
                if v != NONE and int(v) not in seen:
                    seen.add(int(v))
                    nxt.append(int(v))
        frontier = nxt
    assert len(seen) / n >= 0.99


# ---------------------------------------------------------------- Vamana build, hand-worked
#
# Each expected graph below was derived by hand from the two-pass build
# (pass 1 with pruning parameter 1, pass 2 with alpha; per point: GreedySearch
# from the medoid, RobustPrune of visited U current list, then each new
# neighbour j gets the point appended, or, when j's list is full, j's list
# plus the point is pruned again to R).  Squared distances; ties by id.

def _vamana_empty(X, R, Lb, alpha, med, order):
    n = X.shape[0]
    init = np.full((n, R), NONE, np.uint32)
    return oracle.vamana_build(np.asarray(X, np.float32), R, Lb, alpha, med, init,
                               np.asarray(order, np.uint32))


def test_vamana_collinear_alpha1_gives_the_chain():
    # x = 0..4, R = 2, alpha = 1, medoid 2, empty start, order 0..4.
    # Pass 1 ends with rows 0:[2,1] 1:[0,2] 2:[1,3] 3:[2,4] 4:[3]; pass 2
    # prunes every point's candidates (all five points are visited) to its
    # nearest neighbour on each side, nearer first (ties: smaller id).
    X = np.arange(5, dtype=np.float32).reshape(5, 1)
    adj = _vamana_empty(X, 2, 8, 1.0, 2, range(5))
    want = [[1, NONE], [0, 2], [1, 3], [2, 4], [3, NONE]]
    assert adj.tolist() == want


def test_vamana_reverse_edge_overflow_is_pruned():
    # x = 0, 2, 3, 7 (ids 0..3), R = 1, alpha = 1, medoid 1, order 0..3.
    # Pass 1: 0 -> 1 and 1 gets 0; 1 -> 0; 2 -> 1, and 1's full list {0}
    # plus 2 is pruned to its nearer member 2 (d 1 < 4); 3 -> 2 (visited 1,
    # 2), and 2's full list {1} plus 3 is pruned to 1 (d 1 < 16).  Pass 2
    # repeats the same choices: 1's list {2} plus 0 keeps 2, 2's list {1}
    # plus 3 keeps 1.
    X = np.array([[0], [2], [3], [7]], np.float32)
    adj = _vamana_empty(X, 1, 8, 1.0, 1, range(4))
    assert adj.tolist() == [[1], [2], [1], [2]]


def test_vamana_second_pass_keeps_what_the_first_pruned():
    # Points 0:(8,10) 1:(6,10) 2:(8,9) 3:(5,0); squared distances d01 = 4,
    # d02 = 1, d03 = 109, d12 = 5, d13 = 101, d23 = 90.  R = 2, alpha = 1.2,
    # medoid 0, order 1, 2, 3, 0.
    # Pass 1 (parameter 1): 1 -> [0]; 2 -> [0] (1 pruned: d01 = 4 <= d21 = 5);
    # 3 -> [2]; 0 -> [2, 1]; reverse edges make 0:[1,2] then [2,1], 2:[0,3].
    # Pass 2 (alpha^2 = 1.44): 1 -> [0, 3] (1.44 * 109 > 101 keeps 3) and 3
    # gets 1; 2 -> [0, 1] (1.44 * 4 = 5.76 > 5 now keeps 1, the edge pass 1
    # pruned), and 1's full list [0, 3] plus 2 is pruned back to [0, 3];
    # 3 -> [2], and 2's full list [0, 1] plus 3 is pruned to [0, 1]
    # (1.44 * 109 > 90 would keep 3, but R = 2 is reached first); 0 -> [2, 1].
    X = np.array([[8, 10], [6, 10], [8, 9], [5, 0]], np.float32)
    adj = _vamana_empty(X, 2, 8, 1.2, 0, [1, 2, 3, 0])
    assert adj.tolist() == [[2, 1], [0, 3], [0, 1], [2, NONE]]


# ---------------------------------------------------------------- overlapping-shard graph (§2.2)

def _sorted_others(X, i, pool):
    """Members of pool other than i, sorted by (exact squared distance, id)."""
    d = ((X[pool].astype(np.int64) - X[i].astype(np.int64)) ** 2).sum(1)
    keep = [(int(dd), int(p)) for dd, p in zip(d, pool) if p != i]
    return [p for _, p in sorted(keep)]


def test_shard_assignment_is_the_nearest_centres():
    rng = np.random.default_rng(41)
    X = rng.integers(0, 256, size=(500, 6)).astype(np.uint8)
    cen = rng.integers(0, 256, size=(7, 6)).astype(np.float32)
    _, sh = oracle.shard_graph(X, cen, 3, 8, 8, 1.2)
    d = ((X.astype(np.int64)[:, None] - cen.astype(np.int64)[None]) ** 2).sum(-1)
    want = np.argsort(d, axis=1, kind="stable")[:, :3]        # ties: smaller centre index
    assert (sh == want).all()


def test_shard_graph_without_pruning_is_complete_per_shard():
    # alpha huge removes nothing and R >= n - 1, Lb >= n: every shard's
    # subgraph is complete, so a point's row is every other member of its
    # shards, sorted by (distance, id); with ell < S the shards differ.
    rng = np.random.default_rng(42)
    n = 40
    X = np.unique(rng.integers(0, 256, size=(n + 10, 3)), axis=0)[:n].astype(np.uint8)
    X = X[rng.permutation(n)]
    for S, ell in ((1, 1), (2, 2), (3, 2)):
        cen = X[:S].astype(np.float32)
        adj, sh = oracle.shard_graph(X, cen, ell, 40, 64, 1e6, 0.1, 16, iter_cap=200)
        for i in range(n):
            pool = np.where((sh[:, :, None] == sh[i][None, None, :]).any((1, 2)))[0]
            want = _sorted_others(X, i, pool)
            assert adj[i, :len(want)].tolist() == want, (S, ell, i)
            assert (adj[i, len(want):] == NONE).all()


def test_shard_graph_line_alpha1_is_the_chain():
    # one shard, alpha = 1, R = 2, points on a line with distinct gaps: every
    # point keeps its nearest neighbour on each side, nearer first.
    rng = np.random.default_rng(43)
    n = 30
    pos = np.cumsum(rng.integers(1, 5, size=n))
    assert pos.max() < 256
    ids_by_pos = rng.permutation(n)
    X = np.zeros((n, 1), np.uint8)
    X[ids_by_pos, 0] = pos
    adj, _ = oracle.shard_graph(X, X[[ids_by_pos[n // 2]]].astype(np.float32), 1, 2, 64, 1.0, 0.1, 16,
                                iter_cap=200)
    for k in range(n):
        a = ids_by_pos[k]
        nb = sorted((int(pos[j] - pos[k]) ** 2, int(ids_by_pos[j])) for j in (k - 1, k + 1) if 0 <= j < n)
        want = [b for _, b in nb]
        assert adj[a].tolist() == want + [NONE] * (2 - len(want)), (k, adj[a], want)


def test_shard_graph_second_pass_keeps_what_the_first_pruned():
    # One shard centred on point 0 (its entry), insertion 0, 1, 2, 3 one at a
    # time (batch cap 1), R = 2, alpha = 1.2.  Points 0:(0,11) 1:(9,11)
    # 2:(4,1) 3:(6,11); squared distances d01 81, d02 116, d03 36, d12 125,
    # d13 9, d23 104.  Pass 1 (parameter 1): 1 -> [0], 0 gets 1; 2 -> [0]
    # (1 removed: d01 81 <= d21 125), 0 -> [1, 2]; 3 searches 0, 1, 2 and
    # keeps [1, 0]; 1 -> [3, 0]; 0's union {1, 2, 3} is pruned to [3] (3
    # removes 1: 9 <= 81 and 2: 104 <= 116).  Pass 2 (alpha^2 = 1.44): 0 ->
    # [3] (1.44 * 9 <= 81); 1 -> [3] (1.44 * 36 <= 81); 2 -> [3]; 3's union
    # {1, 0, 2} is pruned to [1, 0] (1.44 * 81 > 36 keeps 0, R reached);
    # 3 -> [1, 0].  With alpha in pass 1, 0 would keep 2 (1.44 * 104 > 116).
    X = np.array([[0, 11], [9, 11], [4, 1], [6, 11]], np.float32)
    pos = [oracle.Bloom(16).positions(i) for i in range(4)]
    assert len({p for pp in pos for p in pp}) == 8            # no Bloom false positive
    adj, _ = oracle.shard_graph(X, X[[0]], 1, 2, 8, 1.2, 0.01, 16)
    assert adj.tolist() == [[3, NONE], [3, NONE], [3, NONE], [1, 0]]


def test_shard_graph_invariants():
    rng = np.random.default_rng(44)
    n = 1200
    cen0 = rng.integers(30, 220, size=(5, 8))
    X = np.clip(cen0[rng.integers(0, 5, n)] + rng.normal(0, 20, (n, 8)), 0, 255).astype(np.uint8)
    adj, sh = oracle.shard_graph(X, X[:4].astype(np.float32), 2, 16, 24, 1.2, 0.05, 14)
    for i in range(n):
        row = adj[i]
        ids = row[row != NONE].astype(np.int64)
        assert len(ids) >= 1 and (row[len(ids):] == NONE).all()
        assert i not in ids.tolist() and len(set(ids.tolist())) == len(ids)
        dd = ((X[ids].astype(np.int64) - X[i].astype(np.int64)) ** 2).sum(1)
        assert [(int(a), int(b)) for a, b in zip(dd, ids)] == sorted(zip(dd.tolist(), ids.tolist()))


def test_shard_graph_candidate_pool_is_cut_to_750():
    # nothing pruned (alpha huge), R above 750, every point reachable: each
    # list would hold every other point, but the candidate pool is cut to its
    # 750 nearest (DiskANN's bound), so every row is exactly those.
    rng = np.random.default_rng(45)
    n = 800
    X = np.unique(rng.integers(0, 256, size=(n + 50, 4)), axis=0)[:n].astype(np.uint8)
    X = X[rng.permutation(n)]
    adj, _ = oracle.shard_graph(X, X[:1].astype(np.float32), 1, 790, 1024, 1e6, 0.5, 18,
                                iter_cap=1000)
    for i in range(0, n, 37):
        want = _sorted_others(X, i, np.arange(n))[:750]
        assert adj[i, :750].tolist() == want and (adj[i, 750:] == NONE).all()
