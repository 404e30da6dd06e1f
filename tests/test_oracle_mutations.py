"""Planted mistakes in the oracle must fail its pins.

Each case copies ``oracle/ibs_oracle.c``, plants one plausible mistake (a
wrong condition, a wrong bit order, a dropped factor, a swapped output, a
skipped diagonal), builds it with gcc into a temporary library and runs the
pin tests against it through IBS_ORACLE_LIB.  The pins pass on the real
oracle and must fail on every mutant.  All of this runs on the CPU.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ibs_oracle.c")

MUTATIONS = {
    "ibs0_condition": ("} else if ((a ^ b) == 3) {", "} else if ((a ^ b) == 2) {"),
    "bit_order": ("const int shift = (int)(2 * (s % 4));", "const int shift = (int)(6 - 2 * (s % 4));"),
    "missing_code": ("#define ORACLE_MISSING 1", "#define ORACLE_MISSING 2"),
    "dist_dropped_factor": ("return (double)(c[1] + 2 * (int64_t)c[0]) / (2.0 * (double)c[3]);",
                            "return (double)(c[1] + (int64_t)c[0]) / (2.0 * (double)c[3]);"),
    "swapped_outputs": ("out[0] = (int32_t)ibs0;\n  out[1] = (int32_t)ibs1;",
                        "out[0] = (int32_t)ibs1;\n  out[1] = (int32_t)ibs0;"),
    "skip_needs_both_missing": ("if (a == ORACLE_MISSING || b == ORACLE_MISSING) continue;",
                                "if (a == ORACLE_MISSING && b == ORACLE_MISSING) continue;"),
    "no_diagonal": ("for (int64_t j = i; j < job->n; ++j) {", "for (int64_t j = i + 1; j < job->n; ++j) {"),
}

# Planted mistakes in the linkage-disequilibrium function, run against its own pins.
LD_MUTATIONS = {
    "ld_product_sign": ("(double)(N * Sxy - Sx * Sy)", "(double)(N * Sxy + Sx * Sy)"),
    "ld_missing_not_skipped": ("if (ca == ORACLE_MISSING || cb == ORACLE_MISSING) continue;",
                               "if (ca == ORACLE_MISSING && cb == ORACLE_MISSING) continue;"),
    "ld_fixed_orientation": ("major_a1[k] = hom_a1 >= hom_a2 ? 1 : 0;", "major_a1[k] = 1;"),
    "ld_window_offset": ("const int64_t b = a + 1 + d, slot", "const int64_t b = a + d, slot"),
    "ld_variance_term": ("vx = N * Sxx - Sx * Sx", "vx = N * Sxx - Sx"),
}


# Planted mistakes in the complete-linkage clustering, run against its pins.
CLUSTER_MUTATIONS = {
    "cluster_single_linkage": ("const double d = D[bi * n + k] > D[bj * n + k] ? D[bi * n + k] : D[bj * n + k];",
                               "const double d = D[bi * n + k] < D[bj * n + k] ? D[bi * n + k] : D[bj * n + k];"),
    "cluster_last_tie_wins": ("if (bi < 0 || d < best) {", "if (bi < 0 || d <= best) {"),
    "cluster_id_offset": ("id[bi] = n + step;", "id[bi] = n + step + 1;"),
    "cluster_size_not_added": ("size[bi] += size[bj];", "size[bi] = size[bj];"),
}

# Planted mistakes in the relationship matrix, run against its pins.
GRM_MUTATIONS = {
    "grm_centre_at_p": ("(x_of[a] - 2.0 * p) * (x_of[b] - 2.0 * p) / denom",
                        "(x_of[a] - p) * (x_of[b] - p) / denom"),
    "grm_missing_counted": ("cnt += 1;\n  }\n  return cnt == 0", "}\n  cnt = m;\n  return cnt == 0"),
    "grm_rows_transposed": ("job->out[u * n + k] = oracle_grm_pair(job, j, k);",
                            "job->out[u * n + k] = oracle_grm_pair(job, k, k);"),
    "grm_het_count": ("const double x_of[4] = {2.0, 0.0, 1.0, 0.0};", "const double x_of[4] = {2.0, 0.0, 2.0, 0.0};"),
    "grm_keep_monomorphic": ("if (p <= 0.0 || p >= 1.0) continue;", "if (p < 0.0 || p > 1.0) continue;"),
}

PINS = {**{k: "test_oracle_pins.py" for k in MUTATIONS}, **{k: "test_oracle_ld.py" for k in LD_MUTATIONS},
        **{k: "test_oracle_cluster.py" for k in CLUSTER_MUTATIONS},
        **{k: "test_oracle_grm.py" for k in GRM_MUTATIONS}}
ALL = {**MUTATIONS, **LD_MUTATIONS, **CLUSTER_MUTATIONS, **GRM_MUTATIONS}


@pytest.mark.parametrize("name", sorted(ALL))
def test_planted_mistake_fails_pins(name, tmp_path):
    old, new = ALL[name]
    pins = PINS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_POSIX_C_SOURCE=200809L", "-shared", "-fPIC", "-pthread",
                           str(mutant), "-o", str(lib), "-lm"])
    env = dict(os.environ, IBS_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
