"""Grid refinement of Sec. 4.4 (host logic): the refinement rule of the library and the
oracle's zero-fill regridding (exact for the represented field)."""
import numpy as np
import pytest

import seeded_inputs as si
from oracle import continuation as ct
from oracle.shell import Shell


@pytest.fixture(scope="module")
def rsc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_16635_gb300 import rsc as mod
    return mod


def test_refine_rule(rsc):
    p = rsc.Params(140.0, 1e-5, 1.0, 0.35, 127, 12, 64, 1, 0)
    q, bits = rsc.refine_params(p, 2e-6, 1e-8, 1e-6, 1.2)
    assert bits == 1 and q.Nr == 77 and q.L == 127 and q.Ra == 140.0 and q.Ms == 12
    q, bits = rsc.refine_params(p, 1e-8, 5e-6, 1e-6, 1.2)
    assert bits == 2 and q.L == 153 and q.Nr == 64
    q, bits = rsc.refine_params(p, 1e-3, 1e-3, 1e-6, 1.2)
    assert bits == 3
    q, bits = rsc.refine_params(p, 1e-9, 1e-9, 1e-6, 1.2)
    assert bits == 0 and q.L == 127 and q.Nr == 64
    with pytest.raises(rsc.RscError):
        rsc.refine_params(p, 1e-3, 1e-3, 1e-6, 1.0)


def test_oracle_regrid_is_exact_and_invertible():
    L0, Ms, Nr0, L1, Nr1 = 11, 3, 10, 14, 13
    x = Shell(L0, Ms, Nr0, 1e-3, 100.0).conductive_state() + si.perturbation(L0, Ms, Nr0, seed=9)
    y = ct.regrid(x, L0, Ms, Nr0, L1, Nr1)
    assert np.array_equal(ct.regrid(y, L1, Ms, Nr1, L0, Nr0), x)
    # the represented field is unchanged: same kinetic energy and Nusselt numbers
    s0, s1 = Shell(L0, Ms, Nr0, 1e-3, 100.0), Shell(L1, Ms, Nr1, 1e-3, 100.0)
    assert abs(s0.kinetic_energy(x) - s1.kinetic_energy(y)) < 1e-13 * s0.kinetic_energy(x)
    assert np.allclose(s0.nusselt(x), s1.nusselt(y), rtol=1e-13)
