"""The oracle's pins catch plausible mistakes.

Each case copies the oracle source, plants one mistake of the kind a
restatement of the method could make (a wrong bond, a sign, a power, a
constant, an off-by-one), compiles the copy into a temporary library, and
runs the pins that should catch it against that library in a subprocess
(SGMC_ORACLE_LIB). The case passes only if those pins fail. The unmodified
oracle passes the same pins in the ordinary CPU suite.
"""
import os
import subprocess
import sys

import pytest

from oracle import oracle as orc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MODEL = "tests/test_oracle_model.py"
RNG = "tests/test_oracle_rng_exp.py"
BINS = "tests/test_oracle_bins_hist.py"
CONV = "tests/test_oracle_conventions.py"

# (name, original fragment, planted mistake, pins that must fail)
MUTATIONS = [
    ("local field pairs the -d neighbour with the +d bond",
     "b += J[d * N + im] * (float)s[im];", "b += J[d * N + i] * (float)s[im];",
     [MODEL + "::test_local_field_delta_e_is_energy_difference"]),
    ("field enters dE with the wrong sign",
     "float dE = 2.0f * (float)s[i] * (b + hq);", "float dE = 2.0f * (float)s[i] * (b - hq);",
     [MODEL + "::test_l2_sweep_leaves_boltzmann_stationary"]),
    ("+-J threshold ignores the spin's sign",
     "return thr_t[sb * 7 + u];", "return thr_t[u];",
     [MODEL + "::test_l2_sweep_leaves_boltzmann_stationary"]),
    ("replica exchange with the exponent's sign reversed",
     "float D = cp->db_f[p] * dE;", "float D = -(cp->db_f[p] * dE);",
     [MODEL + "::test_exchange_follows_metropolis_rule_statistics"]),
    ("energy pairs each bond with the wrong neighbour",
     "            int j = neighbour(L, i, d, +1);", "            int j = neighbour(L, i, d, -1);",
     [MODEL + "::test_bond_sum_matches_hamiltonian"]),
    ("a k2 wave vector duplicated instead of (1, -1, 0)",
     "{1, -1, 0}", "{1, 1, 0}",
     [MODEL + "::test_overlap_projections_match_direct_fourier_sum"]),
    ("third moment accumulates Q^2",
     "a[3] += q * q * q;", "a[3] += q * q;",
     [BINS + "::test_histogram_moments_match_accumulators"]),
    ("Taylor coefficient 1/23 instead of 1/24",
     "p = fmaf(p, r, 1.0f / 24.0f);", "p = fmaf(p, r, 1.0f / 23.0f);",
     [RNG + "::test_mc_exp32_error_bound"]),
    ("Philox multiplier off by two",
     "0xD2511F53u", "0xD2511F55u",
     [RNG + "::test_philox_matches_independent_implementation"]),
    ("sweep bin from n instead of n + 1",
     "while (b + 1 < n_bins && ((n + 1) >> (b + 1)) != 0) ++b;",
     "while (b + 1 < n_bins && (n >> (b + 1)) != 0) ++b;",
     [BINS + "::test_bin_populations_closed_form"]),
    ("accumulated energy with the field term's sign reversed",
     "double e = -((double)B[r * nt + t] * qJ + h * (double)M[r * nt + t]);",
     "double e = -((double)B[r * nt + t] * qJ - h * (double)M[r * nt + t]);",
     [MODEL + "::test_high_temperature_energy_follows_the_small_beta_expansion"]),
    ("Metropolis counter without the colour field",
     "((uint32_t)c << 24) | ((uint32_t)r << 16) | tw,",
     "((uint32_t)r << 16) | tw,",
     [CONV + "::test_metropolis_words_differ_between_colours_replicas_slots_and_sites"]),
    ("Metropolis word taken from lane 0 for all four sites of a counter",
     "shi, j & 3);", "shi, 0);",
     [CONV + "::test_metropolis_words_differ_between_colours_replicas_slots_and_sites"]),
    ("Metropolis counter without the replica field",
     "((uint32_t)c << 24) | ((uint32_t)r << 16) | tw,",
     "((uint32_t)c << 24) | tw,",
     [CONV + "::test_metropolis_words_differ_between_colours_replicas_slots_and_sites"]),
    ("exchange always offers the even pairs",
     "exchange_step(&cp, s_base + s, (int)(e & 1), (uint32_t)n,",
     "exchange_step(&cp, s_base + s, 0, (uint32_t)n,",
     [CONV + "::test_exchange_pair_schedule_trace"]),
    ("+-J couplings read lane 0 for every site of a counter",
     "(uint32_t)d, 0u, shi, (i >> 5) & 3);", "(uint32_t)d, 0u, shi, 0);",
     [CONV + "::test_pmj_couplings_are_balanced_and_independent"]),
    ("initial spins drawn without the replica field",
     "((uint32_t)r << 16) | (uint32_t)t, 0u, shi,", "(uint32_t)t, 0u, shi,",
     [CONV + "::test_initial_spins_are_balanced_and_independent"]),
    ("shared slot words keep the slot field",
     "uint32_t tw = cp->slot_shared ? 0u : (uint32_t)t;", "uint32_t tw = (uint32_t)t;",
     [CONV + "::test_slot_shared_words_keep_the_slots_of_a_replica_together"]),
    ("histogram counts disagreeing sites",
     "agree += s0[i] == s1[i];", "agree += s0[i] != s1[i];",
     [BINS + "::test_strong_field_low_temperature_concentrates_at_q_one"]),
]


@pytest.mark.parametrize("name,orig,bad,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_its_pin(tmp_path, name, orig, bad, pins):
    src = open(orc.SRC_PATH).read()
    assert src.count(orig) == 1, "the fragment to mutate must occur exactly once"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(orig, bad))
    lib = orc.compile_oracle(str(mutant), str(tmp_path / "libmutant.so"))
    env = dict(os.environ, SGMC_ORACLE_LIB=lib)
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                          "-m", "not gpu"] + pins, cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=600)
    assert res.returncode == 1, (  # 1: tests ran and at least one failed
        f"planted mistake '{name}' was not caught:\n{res.stdout[-2000:]}")


def test_unmodified_oracle_passes_the_same_pins(tmp_path):
    """Control: the same pins, loaded the same way, pass on a copy of the
    unmodified source."""
    src = tmp_path / "oracle_copy.c"
    src.write_text(open(orc.SRC_PATH).read())
    lib = orc.compile_oracle(str(src), str(tmp_path / "libcopy.so"))
    pins = sorted({p for m in MUTATIONS for p in m[3]})
    env = dict(os.environ, SGMC_ORACLE_LIB=lib)
    res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
                          "-m", "not gpu"] + pins, cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=600)
    assert res.returncode == 0, res.stdout[-2000:]
