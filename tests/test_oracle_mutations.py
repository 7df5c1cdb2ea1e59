"""The oracle's pins must be sensitive: each plausible mistake below, planted in
a scratch copy of the oracle (on the CPU), has to make the pin suite fail."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    "tie_E_before_F": ("(hv == fv ? 2 : 3)", "(hv == ev ? 3 : 2)"),
    "E_extends_on_tie": ("((e_ext > e_open) << 2)", "((e_ext >= e_open) << 2)"),
    "F_extends_on_tie": ("((f_ext > f_open) << 3)", "((f_ext >= f_open) << 3)"),
    "extend_charged_open": ("e_ext = E[at - 1] - e;", "e_ext = E[at - 1] - o;"),
    "transposed_matrix": ("M[c[i - 1] * K + s[j - 1]]", "M[s[j - 1] * K + c[i - 1]]"),
    "last_best_cell": ("if (hv > best) { best = hv;", "if (hv >= best && hv > 0) { best = hv;"),
    "prefix_wrong_slot": ("ins[0] += (uint16_t)(j1 - i1);", "ins[1] += (uint16_t)(j1 - i1);"),
    "suffix_short_by_one": ("for (int32_t t = 1; t <= k; t++) occ[i2 + t] = 1;",
                            "for (int32_t t = 1; t < k; t++) occ[i2 + t] = 1;"),
    "gap_cost_halved": ("+ 2 * g * r;", "+ g * r;"),
    "distance_smaller_self": ("int64_t m = saa > sbb ? saa : sbb;",
                              "int64_t m = saa < sbb ? saa : sbb;"),
    "distance_rounds_up": ("return ORC_ONE - ((int64_t)sab * ORC_ONE) / m;",
                           "return ORC_ONE - ((int64_t)sab * ORC_ONE + m - 1) / m;"),
    "distance_zero_self_far": ("if (m <= 0) return 0;", "if (m <= 0) return ORC_ONE;"),
    "distance_unnormalised": ("sum += orc_distance(S[x * nr + r], self[i], self[ri]);",
                              "sum += (int64_t)self[i] + self[ri] - 2 * (int64_t)S[x * nr + r];"),
    "right_justified": (
        "            for (int32_t u = 0; u < in[j]; u++) row[pos++] = (uint8_t)letters[s[k++]];\n"
        "            for (int32_t u = in[j]; u < G[j]; u++) row[pos++] = '-';\n",
        "            for (int32_t u = in[j]; u < G[j]; u++) row[pos++] = '-';\n"
        "            for (int32_t u = 0; u < in[j]; u++) row[pos++] = (uint8_t)letters[s[k++]];\n"),
    "F_dropped_from_H": ("max2(max2(0, dv), max2(ev, fv));", "max2(max2(0, dv), ev);"),
}


# mistakes in the anchored alignment (the trie path), caught by
# tests/test_oracle_anchored.py
ANCHORED_MUTATIONS = {
    "chain_last_predecessor": ("mp[q] + k <= mp[m] && len[q] + 1 > len[m]",
                               "mp[q] + k <= mp[m] && len[q] + 1 >= len[m]"),
    "anchors_may_overlap": ("mp[q] + k <= mp[m] && len[q] + 1 > len[m]",
                            "mp[q] <= mp[m] && len[q] + 1 > len[m]"),
    "stretch_F_before_diagonal": ("if (H[at] == dv) { occ[a + i] = 1; i--; j--; continue; }",
                                  "if (H[at] == dv && H[at] != F[at]) { occ[a + i] = 1; i--; j--; continue; }"),
    "stretch_edge_gap_uncharged_open": ("F[at] = -(o + (i - 1) * e); H[at] = F[at]; E[at] = ORC_NEG;",
                                        "F[at] = -(i * e); H[at] = F[at]; E[at] = ORC_NEG;"),
}


# mistakes in the fp64 network oracle, caught by tests/test_net_oracle.py
NET_MUTATIONS = {
    "pool_drops_scale": ("dy4 = np.tile(de / np.sqrt(L), (L, 1))", "dy4 = np.tile(de, (L, 1))"),
    "relu_gate_missing": ("dz2 = da2 * (a2 > 0)", "dz2 = da2"),
    "taps_flipped": ("out += xp[k:k + L] @ W[k]", "out += xp[k:k + L] @ W[TAPS - 1 - k]"),
    "adam_no_bias_correction": ("mh = m / (1 - beta1 ** step)", "mh = m"),
}


def _run_mutated(tmp_path, rel_src, old, new, pins, name):
    for d in ("oracle", "seqgen", "tests"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    src = tmp_path / rel_src
    text = src.read_text()
    assert text.count(old) == 1, "mutation site moved: " + name
    src.write_text(text.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        pins], cwd=tmp_path,
                       stdout=subprocess.PIPE, stderr=subprocess.STDOUT, timeout=600)
    assert r.returncode == 1, r.stdout.decode()[-2000:]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    _run_mutated(tmp_path, "oracle/msa_oracle.c", old, new, "tests/test_oracle_pins.py", name)


@pytest.mark.parametrize("name", sorted(ANCHORED_MUTATIONS))
def test_planted_anchored_mistake_is_caught(name, tmp_path):
    old, new = ANCHORED_MUTATIONS[name]
    _run_mutated(tmp_path, "oracle/msa_oracle.c", old, new, "tests/test_oracle_anchored.py", name)


# mistakes in the tree oracle, caught by tests/test_oracle_nj.py
TREE_MUTATIONS = {
    "q_sign_of_r_j": ("Q = (m - 2) * sub - r[:, None] - r[None, :]",
                      "Q = (m - 2) * sub - r[:, None] + r[None, :]"),
    "q_factor_m_minus_1": ("Q = (m - 2) * sub - r[:, None] - r[None, :]",
                           "Q = (m - 1) * sub - r[:, None] - r[None, :]"),
    "pairs_include_diagonal": ("Q[np.tril_indices(m)] = big", "Q[np.tril_indices(m, -1)] = big"),
    "branch_lengths_swapped": ("bl_i = float((m - 2) * dij + int(r[x]) - int(r[y])) / den",
                               "bl_i = float((m - 2) * dij - int(r[x]) + int(r[y])) / den"),
    "update_not_halved": ("(int(D[i, k]) + int(D[j, k]) - dij) >> 1",
                          "(int(D[i, k]) + int(D[j, k]) - dij)"),
    "update_keeps_dij": ("(int(D[i, k]) + int(D[j, k]) - dij) >> 1",
                         "(int(D[i, k]) + int(D[j, k])) >> 1"),
    "gap_columns_compared": ("both = res & res[a]", "both = res | res[a]"),
    "distance_rounds_up": ("(DSCALE * mism) // np.maximum(comp, 1)",
                           "-((-DSCALE * mism) // np.maximum(comp, 1))"),
    "empty_pair_near": ("np.maximum(comp, 1), DSCALE)", "np.maximum(comp, 1), 0)"),
    "cut_smallest_first": ("big = max(cuts, key=lambda v: (len(leaves[v]), -order[v]))",
                           "big = min(cuts, key=lambda v: (len(leaves[v]), -order[v]))"),
    "label_farthest_sample": ("k = min(range(m), key=lambda x: (int(D[i, S[x]]), S[x]))",
                              "k = max(range(m), key=lambda x: (int(D[i, S[x]]), S[x]))"),
    "midpoint_at_a_third": ("half = total / 2.0", "half = total / 3.0"),
    "merged_edge_zero": ("tree[u] = [(walk_s(w), l) for w, l in kids[v]]",
                         "tree[u] = [(walk_s(w), 0.0) for w, l in kids[v]]"),
}


@pytest.mark.parametrize("name", sorted(TREE_MUTATIONS))
def test_planted_tree_mistake_is_caught(name, tmp_path):
    old, new = TREE_MUTATIONS[name]
    _run_mutated(tmp_path, "oracle/nj.py", old, new, "tests/test_oracle_nj.py", name)


@pytest.mark.parametrize("name", sorted(NET_MUTATIONS))
def test_planted_network_mistake_is_caught(name, tmp_path):
    old, new = NET_MUTATIONS[name]
    _run_mutated(tmp_path, "oracle/net.py", old, new, "tests/test_net_oracle.py", name)
