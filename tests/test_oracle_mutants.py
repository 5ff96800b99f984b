"""The pins are sensitive: plausible mistakes planted in a copy of the oracle
(compiled on the CPU into a temporary directory) each fail at least one pin.
The unmodified source passes the same battery."""
from __future__ import annotations

import ctypes
import os
import subprocess

import pytest

from oracle.sivf_oracle import _SRC, bind
from tests import test_golden as golden
from tests import test_oracle_pins as pins

# (name, text in sivf_oracle.c, replacement); every mutant stays memory-safe
MUTANTS = [
    ("ties_to_highest_index", "if (a < 0 || x > bst) {", "if (a < 0 || x >= bst) {"),
    ("own_cluster_not_a_candidate", "if (j == a_prev) x = o->own[i];", "if (j == a_prev) continue;"),
    ("front_back_swapped", "if (o->lambda[j] == 0) mf0[p] += 1; else mf1[p] += 1;",
     "if (o->lambda[j] != 0) mf0[p] += 1; else mf1[p] += 1;",
     "int64_t *pos = (o->lambda[j] == 0) ? &q0[p] : &q1[p];",
     "int64_t *pos = (o->lambda[j] != 0) ? &q0[p] : &q1[p];"),
    ("filtered_scan_truncated", "int64_t e = front ? b + o->if_mf0[s] : o->if_off[s + 1];",
     "int64_t e = front ? b + o->if_mf0[s] / 2 : o->if_off[s + 1];"),
    ("no_unit_length", "nval[d] = w[p] / wn;", "nval[d] = w[p];"),
    ("posting_value_off_by_one", "for (int64_t q = b; q < e; ++q) rho[o->if_cid[q]] += v * o->if_u[q];",
     "for (int64_t q = b; q < e; ++q) rho[o->if_cid[q]] += v * o->if_u[q > b ? q - 1 : q];"),
    ("new_cluster_not_marked_moving", "                o->lambda[a1] = 0;\n", "\n"),
    ("update_objective_of_mean", "snorm[j] = sqrt(ss);", "snorm[j] = sqrt(ss) / (double)cnt;"),
    ("cbicp_branch_inverted", "if (o->lambda[o->if_cid[q]] == 0) rho", "if (o->lambda[o->if_cid[q]] == 1) rho"),
    ("relaxed_test_inverted", "if (rho[a_prev] >= o->own[i]) break;", "if (rho[a_prev] < o->own[i]) break;"),
    ("set_labels_new_cluster_not_moving", "            o->lambda[a1] = 0;\n        }\n    }\n    return 0;",
     "        }\n    }\n    return 0;"),
    ("unfiltered_when_invariant", "int filt = o->icp && a_prev >= 0 && o->own_ok[i] && o->lambda[a_prev] == 1;",
     "int filt = o->icp && a_prev >= 0 && o->own_ok[i] && o->lambda[a_prev] == 0;"),
    ("empty_cluster_zeroed", "nval[d] = o->cen_val[q];", "nval[d] = 0.0;"),
    ("relaxed_tried_always", "2 * n_moving_prev <= k", "n_moving_prev <= k"),
    ("runner_up_not_tracked", "} else if (x > snd) {", "} else if (0) {"),
    ("filtered_counted_as_k", "simcalc += (filt || relax) ? n_moving_prev : k;", "simcalc += k;"),
    ("score_objects_ties_to_highest", "if (rho[j] > bst) { snd = bst; bst = rho[j]; a = j; }",
     "if (rho[j] >= bst) { snd = bst; bst = rho[j]; a = j; }"),
    ("score_objects_runner_up_skips_ties", "else if (rho[j] > snd) snd = rho[j];",
     "else if (rho[j] > snd && rho[j] < bst) snd = rho[j];"),
]


def _battery(lib):
    pins.pin_brute_force(0, False, lib)
    pins.pin_brute_force(1, True, lib)
    pins.pin_update(2, lib)
    pins.pin_layout(3, lib)
    pins.pin_hand_example(lib)
    pins.pin_zero_scores(lib)
    for s in range(4):
        pins.pin_icp_counts(s, lib)
    pins.pin_monotone(21, lib)
    for s in (3, 4):
        pins.pin_cbicp(s, lib)
    pins.pin_relaxed(0, lib)
    pins.pin_set_labels(lib)
    pins.pin_score_objects(0, lib)
    golden.pin_golden(lib)


def _compile(src_text: str, out_dir: str, name: str):
    src = os.path.join(out_dir, f"{name}.c")
    so = os.path.join(out_dir, f"lib{name}.so")
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC", "-o", so, src, "-lm"])
    return bind(ctypes.CDLL(so))


def test_unmodified_oracle_passes_battery(tmp_path):
    with open(_SRC) as f:
        text = f.read()
    _battery(_compile(text, str(tmp_path), "orig"))


@pytest.mark.parametrize("mutant", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, mutant):
    name, edits = mutant[0], mutant[1:]
    with open(_SRC) as f:
        text = f.read()
    for old, new in zip(edits[0::2], edits[1::2]):
        assert text.count(old) == 1, f"mutation anchor for {name} not unique"
        text = text.replace(old, new)
    lib = _compile(text, str(tmp_path), name)
    with pytest.raises(AssertionError):
        _battery(lib)
