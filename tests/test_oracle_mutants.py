"""Plant plausible mistakes in copies of the oracle (CPU only) and check that
the pins in test_oracle_pins.py catch every one of them."""
import os
import subprocess
import sys
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "bang_oracle.c")

# (name, text to replace, replacement, which occurrence (0-based))
MUTANTS = [
    ("adc_table_sign", "float diff = q[o + j] - cc[j];", "float diff = q[o + j] + cc[j];", 0),
    ("adc_table_drops_dim", "for (j = 0; j < ds; j++) {\n                float diff = q[o + j]",
     "for (j = 1; j < ds; j++) {\n                float diff = q[o + j]", 0),
    ("adc_dist_drops_round", "for (h = 4; h >= 1; h >>= 1)", "for (h = 4; h >= 2; h >>= 1)", 0),
    ("adc_dist_wrong_subspace", "T[s * 256 + code[s]]", "T[s * 256 + code[s & ~1u]]", 0),
    ("exact_tree", "r = (j >> 2) & 31u;", "r = j & 31u;", 0),
    ("exact_transposed", "float diff = qf[j] - xf[j];", "float diff = qf[j] - xf[j ^ 1u];", 0),
    ("fnv_prime", "h *= 16777619u;", "h *= 16777617u;", 0),
    ("bloom_one_hash", "pos2[1] = ((uint32_t)(h2 >> 32)", "pos2[1] = pos2[0] | ((uint32_t)0 & (h2 >> 32)", 0),
    ("search_keeps_extra", "nl = (nl + nadd < Lsz) ? nl + nadd : Lsz;",
     "nl = (nl + nadd < Lsz + 1) ? nl + nadd : Lsz + 1;", 0),
    ("rerank_uses_pq", "C[nc].dist = orc_exact_dist(", "C[nc].dist = Lst[u].dist + 0 * orc_exact_dist(", 0),
    ("rerank_list_uses_expanded", "} else if (rerank_list) {", "} else if (0 && rerank_list) {", 0),
    ("rerank_list_uses_pq", "C[nc].dist = orc_exact_dist(q, (const unsigned char *)ix->base + (uint64_t)Lst[i].id",
     "C[nc].dist = Lst[i].dist + 0 * orc_exact_dist(q, (const unsigned char *)ix->base + (uint64_t)Lst[i].id", 0),
    ("rerank_list_drops_last", "        for (i = 0; i < nl; i++) {\n            C[nc].id = Lst[i].id;",
     "        for (i = 0; i + 1 < nl; i++) {\n            C[nc].id = Lst[i].id;", 0),
    ("medoid_no_mean", "for (j = 0; j < d; j++) mean[j] /= (double)n;", "", 0),
    ("kmeans_bad_mean", "sums[c * ds + j] / (double)cnt[c]", "sums[c * ds + j] / (double)(cnt[c] + 1)", 0),
    ("encode_ties_high", "if (acc < best) { best = acc; bc = c; }", "if (acc <= best) { best = acc; bc = c; }", 1),
    ("prune_alpha_unsquared", "double a2 = (double)alpha * (double)alpha;", "double a2 = (double)alpha;", 0),
    ("bruteforce_l1", "ia += t2 * t2;", "ia += t2 < 0 ? -t2 : t2;", 0),
    ("q8_no_offset", "float x = (T[s * 256 + c] - lo[s]) * inv;",
     "float x = (T[s * 256 + c] - 0.0f * lo[s]) * inv;", 0),
    ("q8_truncates", "v = (uint32_t)rintf(x);", "v = (uint32_t)x;", 0),
    ("q8_last_subspace_scale", "if (w > g) g = w;", "g = w;", 0),
    ("q8_search_uses_exact", "if (mode == 2) return (float)orc_adc_dist_q8(",
     "if (mode == 9) return (float)orc_adc_dist_q8(", 0),
    ("cg_kill_strict", "if (lhs <= c[j].dist) dead[j] = 1;", "if (lhs < c[j].dist) dead[j] = 1;", 0),
    ("cg_K_is_Rin", "K = 2 * Rin < m - 1 ? 2 * Rin : m - 1;", "K = Rin < m - 1 ? Rin : m - 1;", 0),
    ("cg_no_reverse_edges", "if (!chose) continue;", "if (1) continue;", 0),
    ("cg_no_repair", "if (indeg[a] != 0 || deg2[a] == 0) continue;", "if (1) continue;", 0),
    ("cg_alpha_unsquared", "float a2 = alpha * alpha;", "float a2 = alpha;", 0),
    ("bf16_truncates", "u += 0x7FFFu + keep_lsb;", "u += 0u * keep_lsb;", 0),
    ("bf16_ties_up", "u += 0x7FFFu + keep_lsb;", "u += 0x8000u + 0u * keep_lsb;", 0),
    ("bf16_mode_uses_f32", "if (mode == 3) orc_adc_table_bf16(T, M, T);", "", 0),
    ("vamana_one_pass", "for (pass = 0; pass < 2; pass++)", "for (pass = 0; pass < 1; pass++)", 0),
    ("vamana_alpha_in_pass1", "float a = pass == 0 ? 1.0f : alpha;", "float a = alpha;", 0),
    ("vamana_no_reverse_edges", "if (has) continue;\n                if (deg < R)",
     "if (has || 1) continue;\n                if (deg < R)", 0),
    ("vamana_overflow_skips",
     "nk = orc_robust_prune(X, d, j, c2, k2, a, R, kept);\n                    for (r = 0; r < R; r++) lj[r] = r < nk ? kept[r] : ORC_NONE;",
     "nk = 0 * k2 + 0 * kept[0];", 0),
    ("vamana_overflow_replaces_last",
     "nk = orc_robust_prune(X, d, j, c2, k2, a, R, kept);\n                    for (r = 0; r < R; r++) lj[r] = r < nk ? kept[r] : ORC_NONE;",
     "nk = 0 * k2 + 0 * kept[0];\n                    lj[R - 1] = p;", 0),
    ("shard_alpha_in_pass1", "float a = pass == 0 ? 1.0f : alpha;\n        uint32_t *start",
     "float a = alpha;\n        uint32_t *start", 0),
    ("shard_no_reverse_edges", "sg_list(vbase, dtype, d, q, c, nc, a, R, 0, vadj + (uint64_t)q * R);",
     "(void)nc;", 0),
    ("shard_merge_one_shard", "for (tt = 0; tt < ell; tt++) {\n            uint32_t vv",
     "for (tt = 0; tt < 1; tt++) {\n            uint32_t vv", 0),
    ("shard_farthest_centres", "best[gg].dist = sg_centre_dist(", "best[gg].dist = -sg_centre_dist(", 0),
    ("shard_farthest_entry", "if (entry[g] == ORC_NONE || dd < bd)", "if (entry[g] == ORC_NONE || dd > bd)", 0),
    ("shard_keeps_repeats", "if (u == 0 || c[i].id != c[u - 1].id) c[u++] = c[i];", "c[u++] = c[i];", 0),
    ("shard_ties_larger_id", "return (a->id < b->id) ? -1 : (a->id > b->id);\n}\n\nstatic float sg_dist",
     "return (a->id > b->id) ? -1 : (a->id < b->id);\n}\n\nstatic float sg_dist", 0),
    ("shard_no_candidate_cap", "if (u > SG_CAND_CAP) u = SG_CAND_CAP;", "", 0),
    ("exact_mode_keeps_rerank", "if (mode == 1) {                    /* Alg. 1",
     "if (mode == 7) {                    /* Alg. 1", 0),
]


def _mutate(src, old, new, occ):
    pos = -1
    for _ in range(occ + 1):
        pos = src.index(old, pos + 1)
    return src[:pos] + new + src[pos + len(old):]


@pytest.mark.parametrize("name,old,new,occ", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new, occ, tmp_path):
    src = open(SRC).read()
    mutated = _mutate(src, old, new, occ)
    assert mutated != src
    c = tmp_path / "mut.c"
    c.write_text(mutated)
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fopenmp", "-I", os.path.join(ROOT, "oracle"), "-o", str(so), str(c),
                           "-lm"])
    env = dict(os.environ, ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(HERE, "test_oracle_pins.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode != 0, "planted mistake %s was not caught:\n%s" % (name, r.stdout[-2000:])
