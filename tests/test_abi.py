"""C-ABI checks that need no GPU: the library loads, exports every function
include/sgmc.h declares, and its host-only entry points behave."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1403_4560_b300 import build as sgbuild
from paper_1403_4560_b300 import inputs, sgmc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    sgbuild.build()
    return sgmc.lib()


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(sg_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_options_default_and_status_strings(lib):
    o = sgmc.default_options()
    assert (o.layout, o.rng_group, o.exchange_every, o.measure_every) == (0, 1, 1, 1)
    assert lib.sg_status_str(sgmc.SG_EINVAL) == b"invalid argument"
    assert lib.sg_status_str(99) == b"unknown status"


def test_options_reject_unknown_names_and_validate_chain_set(lib):
    """Option names are checked by the binding (a misspelt option must not be
    dropped silently), and sg_ensemble_bytes refuses a chain set that is not
    1, 2 or 4 four-slot groups."""
    with pytest.raises(TypeError):
        sgmc.default_options(chain_sets=2)
    o = sgmc.default_options(state_mode=3, chain_set=2)
    assert (o.state_mode, o.chain_set) == (3, 2)
    assert lib.sg_ensemble_bytes(8, 24, 4, sgmc.SG_GAUSS, ctypes.byref(o)) > 0
    for bad in (3, 8, -1):
        o.chain_set = bad
        assert lib.sg_ensemble_bytes(8, 24, 4, sgmc.SG_GAUSS, ctypes.byref(o)) == 0


def test_ensemble_bytes_validates_arguments(lib):
    assert lib.sg_ensemble_bytes(4, 8, 16, 0, None) > 16 * 64 * 16
    assert lib.sg_ensemble_bytes(5, 8, 16, 0, None) == 0   # odd L
    assert lib.sg_ensemble_bytes(4, 0, 16, 0, None) == 0   # no temperatures
    assert lib.sg_ensemble_bytes(4, 8, 0, 0, None) == 0    # no samples
    assert lib.sg_ensemble_bytes(66, 8, 1, 0, None) == 0   # L too large
    assert lib.sg_ensemble_bytes(40, 8, 1, 0, None) > 0    # large L, int8 layout


def test_library_estimators_match_oracle_estimators(lib):
    """Host C++ finalisation (g, chi, xi, R12, jackknife) against the oracle's
    numpy estimators on the same accumulators."""
    L, S, nt = 4, 40, 3
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    J, s0 = inputs.make_instance("pmj", L, S, nt, seed=4)
    st = orc.State(L, T, 0.2, False, seed=9, J=J, spins=s0, n_therm=20)
    st.run(120, threads=4)
    want = orc.observables(st.acc, L)
    got = sgmc.observables_from_acc(st.acc, L)
    for k_lib, k_orc in [("g", "g"), ("chi0", "chi0"), ("chi1", "chi_k1"), ("chi2", "chi_k2"),
                         ("xi", "xi"), ("r12", "r12"), ("e", "e"), ("q2", "q2"), ("q4", "q4")]:
        np.testing.assert_allclose(got[k_lib], want[k_orc], rtol=1e-10, atol=1e-14,
                                   equal_nan=True, err_msg=k_lib)
        np.testing.assert_allclose(got[k_lib + "_err"], want["err"][k_orc], rtol=1e-7,
                                   atol=1e-14, equal_nan=True, err_msg=k_lib + "_err")
