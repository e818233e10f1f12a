"""Planted mistakes in copies of the oracle: the pin suite must catch every one.

The oracle is trusted because its pins (tests/test_oracle_pins.py) tie it to values
the paper and the mathematics fix.  Here each plausible mistake -- a dropped term, a
wrong index or comparison, a transposed operand -- is planted in a copy of the
oracle on the CPU, and the pin suite, run against that copy, must fail.  The
unchanged copy must pass, so a failure means the mistake was caught, not that the
harness broke."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

from conftest import ROOT

ORACLE = os.path.join(ROOT, "oracle")

# (name, file, text in the oracle, planted replacement)
MUTANTS = [
    # Philox4x32-10
    ("philox_operands_transposed", "pbn_oracle.c",
     "uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;", "uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x2;"),
    ("philox_key_not_bumped", "pbn_oracle.c", "        k0 += 0x9E3779B9u;\n", ""),
    ("philox_nine_rounds", "pbn_oracle.c", "for (int round = 0; round < 10; ++round)",
     "for (int round = 0; round < 9; ++round)"),
    ("counter_traj_step_swapped", "pbn_oracle.c",
     "ctr[0] = (uint32_t)(traj & 0xFFFFFFFFu);\n    ctr[1] = (uint32_t)(step & 0xFFFFFFFFu);",
     "ctr[0] = (uint32_t)(step & 0xFFFFFFFFu);\n    ctr[1] = (uint32_t)(traj & 0xFFFFFFFFu);"),
    # perturbation draws (PERT, GEO) and thresholds
    # (u <= P for u < P changes the rate by 2^-32: no sample of feasible size sees it)
    ("pert_threshold_half_scale", "pbn_oracle.c", "static uint64_t pert_threshold(double p) { return (uint64_t)floor(p * 4294967296.0); }",
     "static uint64_t pert_threshold(double p) { return (uint64_t)floor(p * 2147483648.0); }"),
    ("pert_level_halves_swapped", "pbn_oracle.c",
     "level[2 * h] = ((uint64_t)x[1] << 32) | x[0];", "level[2 * h] = ((uint64_t)x[0] << 32) | x[1];"),
    ("pert_levels_lsb_first", "pbn_oracle.c", "u |= ((level[l] >> b) & 1u) << (31 - l);",
     "u |= ((level[l] >> b) & 1u) << l;"),
    ("geo_threshold_limb_off_by_one", "pbn_oracle.c", "const int drop = k - 1; /* limbs shifted out */",
     "const int drop = k; /* limbs shifted out */"),
    ("geo_word_halves_swapped", "pbn_oracle.c",
     "uint64_t U = (w % 2 == 0) ? (((uint64_t)x[1] << 32) | x[0]) : (((uint64_t)x[3] << 32) | x[2]);",
     "uint64_t U = (w % 2 == 1) ? (((uint64_t)x[1] << 32) | x[0]) : (((uint64_t)x[3] << 32) | x[2]);"),
    # selection
    ("sel_cumulative_sum_dropped", "pbn_oracle.c", "        C = C + nd->f[j - 1].c;\n        double v",
     "        C = nd->f[j - 1].c;\n        double v"),
    ("sel_slot_lane_shifted", "pbn_oracle.c", "uint64_t u = x[r & 3];", "uint64_t u = x[(r + 1) & 3];"),
    ("sel_rank_over_all_nodes", "pbn_oracle.c", "cx->rank[i] = g->node[i].nf >= 2 ? r++ : -1;",
     "cx->rank[i] = g->node[i].nf >= 2 ? r++ : (r++, -1);"),
    # initial state and the step of Eq. 1
    ("init_word_halves_swapped", "pbn_oracle.c",
     "keyed_block(seed, traj, 0, DOM_INIT, (uint32_t)w >> 1, x);\n        uint64_t word = (w % 2 == 0)",
     "keyed_block(seed, traj, 0, DOM_INIT, (uint32_t)w >> 1, x);\n        uint64_t word = (w % 2 == 1)"),
    ("eq1_flip_as_or", "pbn_oracle.c", "for (int i = 0; i < n; ++i) s[i] ^= gam[i];",
     "for (int i = 0; i < n; ++i) s[i] |= gam[i];"),
    ("eq1_perturbed_step_applies_functions", "pbn_oracle.c",
     "            } else if (draw_pert(cx, jb->seed, traj, t, gam)) {\n                for (int i = 0; i < n; ++i) s[i] ^= gam[i];\n            } else {",
     "            } else {\n                draw_pert(cx, jb->seed, traj, t, gam);"),
    ("function_inputs_reversed", "pbn_oracle.c", "x |= (uint64_t)s[f->par[b]] << b;",
     "x |= (uint64_t)s[f->par[b]] << (f->k - 1 - b);"),
    ("nodewise_flip_keeps_value", "pbn_oracle.c", "s2[i] = gam[i] ? (uint8_t)(s[i] ^ 1u) :", "s2[i] = gam[i] ? s[i] :"),
    ("eq1_functions_read_the_new_state", "pbn_oracle.c",
     "for (int i = 0; i < n; ++i) s2[i] = (uint8_t)eval_fun(&g->node[i].f[ch[i]], s);\n                memcpy(s, s2, (size_t)n);\n            }\n            int z",
     "for (int i = 0; i < n; ++i) s[i] = (uint8_t)eval_fun(&g->node[i].f[ch[i]], s);\n            }\n            int z"),
    # the network text
    ("hex_digits_read_most_significant_first", "pbn_oracle.c", "int v = hexval(th[nd_hex - 1 - d]);",
     "int v = hexval(th[d]);"),
    # counts of the two-state chain
    ("pair_counts_transposed", "pbn_oracle.c", "cnt[1 + 2 * z_prev + z] += 1;", "cnt[1 + z_prev + 2 * z] += 1;"),
    ("meta_values_ignored", "pbn_oracle.c", "if (s[jb->meta_ids[m]] != jb->meta_vals[m]) return 0;",
     "if (s[jb->meta_ids[m]] != 1) return 0;"),
    ("first_state_not_counted", "pbn_oracle.c",
     "        if (!jb->init_states && jb->step_begin >= jb->count_from) cnt[0] += (uint64_t)z_prev;\n", ""),
    ("resumed_run_recounts_its_initial_state", "pbn_oracle.c",
     "if (!jb->init_states && jb->step_begin >= jb->count_from) cnt[0] += (uint64_t)z_prev;",
     "if (jb->step_begin == jb->count_from) cnt[0] += (uint64_t)z_prev;"),
    ("visit_window_off_by_one", "pbn_oracle.c", "if (t + 1 >= jb->count_from) cnt[0] += (uint64_t)z;",
     "if (t >= jb->count_from) cnt[0] += (uint64_t)z;"),
    # exact transition matrix
    ("nodewise_matrix_flip_toward_value", "pbn_oracle.c",
     "q1[i] = pe * (double)(st[i] ^ 1u) + (1.0 - pe) * q1[i];", "q1[i] = pe * (double)st[i] + (1.0 - pe) * q1[i];"),
    ("matrix_unperturbed_counted_twice", "pbn_oracle.c", "if (semantics == 0 && s2 != s) row[s2]",
     "if (semantics == 0) row[s2]"),
    ("matrix_choice_interval_index", "pbn_oracle.c",
     "uint64_t hi = j == nd->nf - 1 ? ((uint64_t)1 << 32) : T[j + 1];",
     "uint64_t hi = j == nd->nf - 1 ? ((uint64_t)1 << 32) : T[j];"),
    # Definition 1 and the reachability variant
    ("leaves_self_edges_counted", "pbn_oracle.c",
     "                if (v != u) child[(size_t)v * n + u] = 1;\n            }\n    memset(is_leaf",
     "                child[(size_t)v * n + u] = 1;\n            }\n    memset(is_leaf"),
    ("reach_edges_reversed", "pbn_oracle.c", "if (child[(size_t)v * n + u] && keep[u])",
     "if (child[(size_t)u * n + v] && keep[u])"),
    ("leaves_interest_ignored", "pbn_oracle.c", "if (is_leaf[v] || intr[v]) continue;", "if (is_leaf[v]) continue;"),
    ("reach_interest_not_kept", "pbn_oracle.c", "        keep[interest[m]] = 1;\n", ""),
    # the two-state chain estimator and the stationary distribution (numpy side)
    ("estimate_beta_wrong_count", "oracle.py", "b = n10 / (n10 + n11)", "b = n11 / (n10 + n11)"),
    ("estimate_sample_size_power", "oracle.py", "nreal = a * b * (2.0 - a - b) / (a + b) ** 3",
     "nreal = a * b * (2.0 - a - b) / (a + b) ** 2"),
    ("estimate_burn_in_min_for_max", "oracle.py", "eps * (a + b) / max(a, b)", "eps * (a + b) / min(a, b)"),
    ("estimate_initial_states_dropped", "oracle.py", "L = n00 + n01 + n10 + n11 + int(n_traj)",
     "L = n00 + n01 + n10 + n11"),
    ("stationary_transposed", "oracle.py", "nxt = pi @ M", "nxt = M @ pi"),
    ("estimate_mixing_rate_signed", "oracle.py", "lam = abs(1.0 - a - b)", "lam = 1.0 - a - b"),
]


def _copy(dst, name=None):
    """A copy of the oracle in dst, with mutant `name` planted (None: unchanged)."""
    os.makedirs(dst)
    for f in ("oracle.py", "pbn_oracle.c"):
        shutil.copy(os.path.join(ORACLE, f), os.path.join(dst, f))
    if name is None:
        return
    _, fname, old, new = next(m for m in MUTANTS if m[0] == name)
    path = os.path.join(dst, fname)
    src = open(path).read()
    assert src.count(old) == 1, f"{name}: the planted text must occur exactly once"
    open(path, "w").write(src.replace(old, new))


def _pins(dst):
    """Run the pin suite against the oracle copy in dst: (return code, output tail)."""
    env = dict(os.environ, PBN_ORACLE_DIR=dst)
    p = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return p.returncode, (p.stdout + p.stderr)[-1500:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    base = tmp_path_factory.mktemp("oracle_mutants")
    names = [None] + [m[0] for m in MUTANTS]
    dirs = {}
    for nm in names:
        d = str(base / (nm or "unchanged"))
        _copy(d, nm)
        dirs[nm] = d
    with ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        res = dict(zip(names, ex.map(lambda nm: _pins(dirs[nm]), names)))
    return res


def test_unchanged_copy_passes_the_pins(outcomes):
    rc, tail = outcomes[None]
    assert rc == 0, tail


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(outcomes, name):
    rc, tail = outcomes[name]
    # 1: some pin failed (not a collection or usage error)
    assert rc == 1 and "failed" in tail, tail
