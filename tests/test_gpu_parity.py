"""GPU (CUDA, through the C ABI) against the FP64 oracle on the same seeded inputs.

Every comparison is element by element: per field (e, f, T) the largest difference over
the largest entry of the oracle's field, max |got - want| / max |want|.  Fixed bounds:
  * transform pipeline (explicit terms): 1e-12;
  * FP64 step and Jacobian action: 1e-11 (the per-step bound of the FP64 path);
  * FP64 implicit solve (rsc_implicit_solve, Sec. 3.2): row-scaled backward error of the
    oracle's assembled chain system below 64 u (u = 2^-53), solution within 1e-11 of the
    oracle's; the double-float solve of the mixed path: 64 u_df (u_df = 2^-48, the
    precision of its split tables) and 32 x 1e-11;
  * converged rotating waves: 1e-10 (FP64), drift within 1e-8 (mixed).
Both sides solve the chains after row equilibration (the oracle's banded LU, the library's
block factorisation), which is what lets two independent FP64 codes agree to 1e-11 on the
low-Ekman chains: unscaled, the boundary rows lost up to 1e-8 to pivoting against rows
13 orders of magnitude larger.
"""
import functools

import numpy as np
import pytest

import seeded_inputs as si
from oracle.shell import Shell

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53        # unit roundoff of FP64
U48 = 2.0 ** -48        # of the double-float (FP32 hi + lo) tables of the mixed chain solve


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return _t


def _maxabs_fields(s, got, want):
    """Per field: max |got - want| / max |want| over its complex coefficients."""
    g = s.to_complex(got)
    w = s.to_complex(want)
    return [float(np.abs(g[i] - w[i]).max() / max(float(np.abs(w[i]).max()), 1e-300))
            for i in range(3)]


def _rel(got, want):
    return float(np.abs(got - want).max() / np.abs(want).max())


CASES = [
    # name, L, Ms, Nr, Ek, Ra
    ("tiny", 7, 4, 10, 1e-3, 80.0),
    ("ragged", 13, 3, 17, 3e-3, 95.0),      # odd Nr, m not dividing L, nlat2 not a warp multiple
    ("one_m", 9, 9, 12, 1e-3, 60.0),        # m in {0, L}
    ("C1", 31, 4, 24, 1e-3, 120.0),
]
C3 = ("C3", 127, 12, 64, 1e-5, 140.0)       # the low-Ekman configuration of the benchmark
CASES_C3 = CASES + [C3]

_SHELLS = {}


def _shell(L, Ms, Nr, Ek, Ra, coriolis="implicit"):
    """One oracle Shell per configuration (its factorisations are cached inside)."""
    key = (L, Ms, Nr, Ek, Ra, coriolis)
    if key not in _SHELLS:
        _SHELLS[key] = Shell(L, Ms, Nr, Ek, Ra, coriolis=coriolis)
    return _SHELLS[key]


@functools.lru_cache(maxsize=None)
def _oracle_step(L, Ms, Nr, Ek, Ra, seed, amp, C, dt, nsteps):
    s = _shell(L, Ms, Nr, Ek, Ra)
    x = s.conductive_state() + si.perturbation(L, Ms, Nr, seed=seed, amp=amp)
    return x, s.step(x, C, dt, nsteps=nsteps)


@functools.lru_cache(maxsize=None)
def _oracle_jvp(L, Ms, Nr, Ek, Ra, seed, with_drift, C, dt):
    s = _shell(L, Ms, Nr, Ek, Ra)
    U = s.conductive_state() + si.perturbation(L, Ms, Nr, seed=seed, amp=3e-2)
    u = si.random_vector(L, Ms, Nr, seed=seed + 1)
    J = s.real_index("T", Ms, Ms, 1, 1) if with_drift else None
    if with_drift:
        u[J] = 0.7
    return U, u, J, s.jvp(U, C, J, u, dt)


@pytest.mark.parametrize("name,L,Ms,Nr,Ek,Ra", CASES_C3)
def test_explicit_terms_parity(torch, name, L, Ms, Nr, Ek, Ra):
    from paper_2508_16635_gb300 import RotatingShell
    s = _shell(L, Ms, Nr, Ek, Ra)
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra)
    x = s.conductive_state() + si.perturbation(L, Ms, Nr, seed=21, amp=3e-2)
    got = gpu.explicit_terms(torch.tensor(x, device="cuda")).cpu().numpy()
    want = s.to_real(s.explicit_terms(s.to_complex(x)))
    errs = _maxabs_fields(s, got, want)
    assert max(errs) < 1e-12, errs
    gpu.close()


@pytest.mark.parametrize("name,L,Ms,Nr,Ek,Ra", CASES_C3)
@pytest.mark.parametrize("dt,C", [(1e-4, 0.0), (2e-3, -2.7), (200.0, 1.3)])
def test_step_parity(torch, name, L, Ms, Nr, Ek, Ra, dt, C):
    from paper_2508_16635_gb300 import RotatingShell
    x, want = _oracle_step(L, Ms, Nr, Ek, Ra, 22, 1e-2, C, dt, 2)
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra)
    U = torch.tensor(x, device="cuda")
    gpu.step(U, C, dt, nsteps=2)
    errs = _maxabs_fields(_shell(L, Ms, Nr, Ek, Ra), U.cpu().numpy(), want)
    assert max(errs) < 1e-11, errs
    gpu.close()


def test_step_host_buffer_matches_device_step(torch):
    from paper_2508_16635_gb300 import RotatingShell
    L, Ms, Nr = 15, 4, 16
    gpu = RotatingShell(L, Ms, Nr, 1e-3, 100.0)
    x = np.ascontiguousarray(gpu.conductive_state().cpu().numpy() + si.perturbation(L, Ms, Nr, 5))
    U = torch.tensor(x, device="cuda")
    gpu.step(U, 0.5, 1e-3, nsteps=3)
    h = x.copy()
    gpu.step_host(h, 0.5, 1e-3, nsteps=3)
    assert np.array_equal(h, U.cpu().numpy())
    gpu.close()


@pytest.mark.parametrize("name,L,Ms,Nr,Ek,Ra", CASES_C3)
@pytest.mark.parametrize("with_drift", [False, True])
def test_jacobian_parity(torch, name, L, Ms, Nr, Ek, Ra, with_drift):
    from paper_2508_16635_gb300 import RotatingShell
    C, dt = -1.1, 200.0
    U, u, J, want = _oracle_jvp(L, Ms, Nr, Ek, Ra, 23, with_drift, C, dt)
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra)
    got = gpu.apply_jacobian(torch.tensor(U, device="cuda"), C, J,
                             torch.tensor(u, device="cuda"), dt).cpu().numpy()
    errs = _maxabs_fields(_shell(L, Ms, Nr, Ek, Ra), got, want)
    assert max(errs) < 1e-11, errs
    gpu.close()


# N_r = 96 reaches the compile-time (96, 144) instantiation of the FP32 radial kernels
CASES_MIXED_JVP = CASES_C3 + [("Nr96", 15, 4, 96, 1e-3, 80.0)]


@pytest.mark.parametrize("name,L,Ms,Nr,Ek,Ra", CASES_MIXED_JVP)
@pytest.mark.parametrize("with_drift", [False, True])
def test_mixed_jacobian_parity(torch, name, L, Ms, Nr, Ek, Ra, with_drift):
    """Mixed path: the Jacobian action (FP32 radial evaluation, transforms, products and
    right-hand side; double-float chain solve) against the FP64 oracle, field by field.
    The bound is FP32-level: sums of O(100) terms rounded to FP32 (unit roundoff 6e-8) and
    3xTF32 Legendre products, about 1e-6 of the field magnitudes (measured on a GB300: at
    most 1.6e-6 over these cases); a missing or wrong term (a boundary row, the drift term,
    a Coriolis coupling) is O(1)."""
    from paper_2508_16635_gb300 import RotatingShell
    C, dt = -1.1, 200.0
    U, u, J, want = _oracle_jvp(L, Ms, Nr, Ek, Ra, 29, with_drift, C, dt)
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra, precision="mixed")
    got = gpu.apply_jacobian(torch.tensor(U, device="cuda"), C, J,
                             torch.tensor(u, device="cuda"), dt).cpu().numpy()
    errs = _maxabs_fields(_shell(L, Ms, Nr, Ek, Ra), got, want)
    assert max(errs) < 1e-5, errs
    gpu.close()


def test_jacobian_batch_of_directions(torch):
    from paper_2508_16635_gb300 import RotatingShell
    L, Ms, Nr = 15, 4, 16
    s = Shell(L, Ms, Nr, 1e-3, 120.0)
    gpu = RotatingShell(L, Ms, Nr, 1e-3, 120.0)
    U = s.conductive_state() + si.perturbation(L, Ms, Nr, seed=31, amp=3e-2)
    us = np.stack([si.random_vector(L, Ms, Nr, seed=40 + q) for q in range(3)])
    got = gpu.apply_jacobian(torch.tensor(U, device="cuda"), 0.2, None,
                             torch.tensor(us.reshape(-1), device="cuda"), 200.0).cpu().numpy()
    for q in range(3):
        assert _rel(got[q * s.n:(q + 1) * s.n], s.jvp(U, 0.2, None, us[q], 200.0)) < 1e-10
    gpu.close()


LARGE = [("C3-ish", 127, 12, 24, 1e-5, 140.0), ("L255", 255, 16, 8, 3e-6, 200.0),
         ("L255-Ms8", 255, 8, 12, 3e-6, 200.0)]


@pytest.mark.parametrize("name,L,Ms,Nr,Ek,Ra", LARGE)
def test_explicit_terms_parity_large_truncations(torch, name, L, Ms, Nr, Ek, Ra):
    """The FP64 transform pipeline at the largest truncations (the C5 degree L = 255), at the
    same fixed bound as the small cases: both sides' quadrature weights and Legendre tables
    are correct to the last bit (the oracle's round trip is pinned at 1e-13 up to L = 255)."""
    from paper_2508_16635_gb300 import RotatingShell
    s = _shell(L, Ms, Nr, Ek, Ra)
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra)
    x = s.conductive_state() + si.perturbation(L, Ms, Nr, seed=29, amp=3e-2)
    got = gpu.explicit_terms(torch.tensor(x, device="cuda")).cpu().numpy()
    want = s.to_real(s.explicit_terms(s.to_complex(x)))
    errs = _maxabs_fields(s, got, want)
    assert max(errs) < 1e-12, errs
    gpu.close()


@pytest.mark.parametrize("name,L,Ms,Nr,Ek,Ra", CASES_C3 + LARGE)
def test_mixed_explicit_terms_accuracy(torch, name, L, Ms, Nr, Ek, Ra):
    """Mixed path: FP32 radial evaluation, tensor-core (3xTF32) Legendre synthesis, FP32 DFT,
    products and analysis; the explicit terms agree with the FP64 oracle to FP32 accuracy."""
    from paper_2508_16635_gb300 import RotatingShell
    s = _shell(L, Ms, Nr, Ek, Ra)
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra, precision="mixed")
    x = s.conductive_state() + si.perturbation(L, Ms, Nr, seed=28, amp=3e-2)
    got = gpu.explicit_terms(torch.tensor(x, device="cuda")).cpu().numpy()
    want = s.to_real(s.explicit_terms(s.to_complex(x)))
    errs = _maxabs_fields(s, got, want)
    assert max(errs) < 2e-5, errs
    gpu.close()


@pytest.mark.parametrize("name,L,Ms,Nr,Ek,Ra", CASES_C3 + LARGE)
def test_tensor_core_analysis_accuracy(torch, name, L, Ms, Nr, Ek, Ra):
    """Mixed path with the tensor-core Legendre analysis (tcgen05, 3xTF32; analysis_tc = 1):
    the explicit terms agree with the FP64 oracle to FP32 accuracy, like the CUDA-core one."""
    from paper_2508_16635_gb300 import RotatingShell
    s = _shell(L, Ms, Nr, Ek, Ra)
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra, precision="mixed")
    gpu.set_tuning(dict(gpu.tuning(), analysis_tc=1))
    x = s.conductive_state() + si.perturbation(L, Ms, Nr, seed=28, amp=3e-2)
    got = gpu.explicit_terms(torch.tensor(x, device="cuda")).cpu().numpy()
    want = s.to_real(s.explicit_terms(s.to_complex(x)))
    errs = _maxabs_fields(s, got, want)
    assert max(errs) < 2e-5, errs
    gpu.close()


def test_mixed_precision_step_error(torch):
    from paper_2508_16635_gb300 import RotatingShell
    L, Ms, Nr, Ek, Ra = 31, 4, 24, 1e-3, 120.0
    s = Shell(L, Ms, Nr, Ek, Ra)
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra, precision="mixed")
    x = s.conductive_state() + si.perturbation(L, Ms, Nr, seed=25, amp=1e-2)
    U = torch.tensor(x, device="cuda")
    gpu.step(U, 0.0, 1e-3)
    want = s.step(x, 0.0, 1e-3)
    # only the explicit part is FP32: compare the change of the state
    err = np.linalg.norm(U.cpu().numpy() - want) / np.linalg.norm(want - x)
    assert err < 1e-4
    gpu.close()


def _rw_initial_guess(s, M, nsteps=400, dt=2e-3):
    """Oracle time stepping from an m = M temperature seed (the paper starts from cos(M phi))."""
    x = s.to_complex(s.conductive_state())
    prof = 1e-2 * np.sin(np.pi * (s.rc - s.r_in))
    x[2, s.pair_index(M, M)] += np.linalg.solve(s.E[0], prof)
    U = s.step(s.to_real(x), 0.0, dt, nsteps=nsteps)
    U1 = s.step(U, 0.0, dt, nsteps=5)
    from oracle import krylov
    return U, krylov.drift_estimate(s, U, U1, 5 * dt, M), krylov.phase_index(s, U, M)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_newton_rotating_wave_parity(torch, precision):
    """RW4 at Ek = 1e-3, Ra = 120 (Table 1 row 1) on a reduced truncation: the GPU Newton-GMRES
    solution matches the oracle's to 1e-10 (FP64) and the drift to 1e-8 (mixed)."""
    from oracle import krylov
    from paper_2508_16635_gb300 import RotatingShell
    L, Ms, Nr, Ek, Ra = 23, 4, 20, 1e-3, 120.0
    s = Shell(L, Ms, Nr, Ek, Ra)
    U0, C0, J = _rw_initial_guess(s, 4)
    Uo, Co, hist = krylov.newton(s, U0, C0, J, dt=200.0, tol=1e-11, max_newton=12, kmax=120)
    assert hist[-1]["residual"] < 1e-11
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra, precision=precision)
    U = torch.tensor(U0, device="cuda")
    C, rep, st = gpu.newton_rw(U, C0, J, tol=1e-11, max_newton=14, kmax=120, gmres_tol=1e-10)
    assert st == 0, rep
    Ug = U.cpu().numpy()
    if precision == "fp64":
        assert _rel(Ug, Uo) < 1e-10
        assert abs(C - Co) < 1e-10 * abs(Co)
    else:
        assert _rel(Ug, Uo) < 1e-9
        assert abs(C - Co) < 1e-8 * abs(Co)
    gpu.close()


# ---- explicit-Coriolis variant (Eqs. expcor_e/f), the comparison scheme of Sec. 5 ----------
@pytest.mark.parametrize("name,L,Ms,Nr,Ek,Ra", CASES[:2] + CASES[3:])
def test_explicit_coriolis_step_and_jacobian_parity(torch, name, L, Ms, Nr, Ek, Ra):
    from paper_2508_16635_gb300 import RotatingShell
    s = _shell(L, Ms, Nr, Ek, Ra, coriolis="explicit")
    x = s.conductive_state() + si.perturbation(L, Ms, Nr, seed=26, amp=1e-2)
    want = s.step(x, 0.7, 1e-3, nsteps=2)
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra, coriolis="explicit")
    U = torch.tensor(x, device="cuda")
    gpu.step(U, 0.7, 1e-3, nsteps=2)
    errs = _maxabs_fields(s, U.cpu().numpy(), want)
    assert max(errs) < 1e-11, errs
    u = si.random_vector(L, Ms, Nr, seed=27)
    J = s.real_index("T", Ms, Ms, 1, 1)
    u[J] = -0.4
    want = s.jvp(x, 0.7, J, u, 200.0)
    got = gpu.apply_jacobian(torch.tensor(x, device="cuda"), 0.7, J,
                             torch.tensor(u, device="cuda"), 200.0).cpu().numpy()
    errs = _maxabs_fields(s, got, want)
    assert max(errs) < 1e-11, errs
    gpu.close()


def test_explicit_and_implicit_coriolis_reach_the_same_wave_on_the_gpu(torch):
    """Eq. finalrhs: the root of B - I does not depend on how L is split, so both schemes
    converge to the same rotating wave; the implicit one in fewer Jacobian actions (Sec. 5)."""
    from paper_2508_16635_gb300 import RotatingShell
    L, Ms, Nr, Ek, Ra = 23, 4, 20, 1e-3, 120.0
    s = Shell(L, Ms, Nr, Ek, Ra)
    U0, C0, J = _rw_initial_guess(s, 4)
    res = {}
    for mode in ("implicit", "explicit"):
        gpu = RotatingShell(L, Ms, Nr, Ek, Ra, coriolis=mode)
        U = torch.tensor(U0, device="cuda")
        C, rep, st = gpu.newton_rw(U, C0, J, tol=1e-11, max_newton=14, kmax=400, gmres_tol=1e-10)
        assert st == 0, (mode, rep)
        res[mode] = (U.cpu().numpy(), C, rep["gmres_total"])
        gpu.close()
    Ui, Ci, gi = res["implicit"]
    Ue, Ce, ge = res["explicit"]
    assert _rel(Ue, Ui) < 1e-8 and abs(Ce - Ci) < 1e-8 * abs(Ci)
    assert ge > gi


@pytest.mark.parametrize("name,L,Ms,Nr,Ek,Ra", CASES)
def test_diagnostics_parity(torch, name, L, Ms, Nr, Ek, Ra):
    """rsc_diagnostics (Parseval on the GPU) against the oracle's grid quadrature."""
    from paper_2508_16635_gb300 import RotatingShell
    s = Shell(L, Ms, Nr, Ek, Ra)
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra)
    x = s.conductive_state() + si.perturbation(L, Ms, Nr, seed=33, amp=3e-2)
    ke, nu_in, nu_out = gpu.diagnostics(torch.tensor(x, device="cuda"))
    ke_o = s.kinetic_energy(x)
    nu_in_o, nu_out_o = s.nusselt(x)
    assert abs(ke - ke_o) < 1e-11 * ke_o
    assert abs(nu_in - nu_in_o) < 1e-11 * abs(nu_in_o)
    assert abs(nu_out - nu_out_o) < 1e-11 * abs(nu_out_o)
    cond = s.conductive_state()
    ke0, n0, n1 = gpu.diagnostics(torch.tensor(cond, device="cuda"))
    c_in, c_out = s.nusselt(cond)       # 1 up to the N_r truncation of the 1/r profile
    assert ke0 == 0.0 and abs(n0 - c_in) < 1e-11 and abs(n1 - c_out) < 1e-11
    gpu.close()


@pytest.mark.parametrize("name,L,Ms,Nr,Ek,Ra", CASES)
@pytest.mark.parametrize("coriolis", ["implicit", "explicit"])
def test_step2_parity(torch, name, L, Ms, Nr, Ek, Ra, coriolis):
    """Second-order step (Crank-Nicolson + Heun): the GPU's half-step form against the
    oracle's direct Crank-Nicolson form, FP64, from a state that meets the BCs.  The GPU
    forms x' = 2 y - x from the half-step solution y, which doubles the solve's rounding
    relative to the oracle's direct solve: twice the step bound."""
    from paper_2508_16635_gb300 import RotatingShell
    s = _shell(L, Ms, Nr, Ek, Ra, coriolis=coriolis)
    dt = 2e-4
    x = s.step(s.conductive_state() + si.perturbation(L, Ms, Nr, seed=24, amp=1e-2), 0.0, dt)
    want = s.step2(x, dt, nsteps=2)
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra, coriolis=coriolis)
    U = torch.tensor(x, device="cuda")
    gpu.step2(U, dt, nsteps=2)
    errs = _maxabs_fields(s, U.cpu().numpy(), want)
    assert max(errs) < 2e-11, errs
    gpu.close()


def test_step2_mixed_precision_error(torch):
    """The mixed path's second-order step (FP32 transforms) stays within 1e-5 of the oracle."""
    from paper_2508_16635_gb300 import RotatingShell
    L, Ms, Nr, Ek, Ra = 31, 4, 24, 1e-3, 120.0
    s = Shell(L, Ms, Nr, Ek, Ra)
    dt = 2e-4
    x = s.step(s.conductive_state() + si.perturbation(L, Ms, Nr, seed=25, amp=1e-2), 0.0, dt)
    want = s.step2(x, dt, nsteps=3)
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra, precision="mixed")
    U = torch.tensor(x, device="cuda")
    gpu.step2(U, dt, nsteps=3)
    errs = _maxabs_fields(s, U.cpu().numpy(), want)
    assert max(errs) < 1e-5, errs
    gpu.close()


def test_ra_continuation_parity(torch):
    """rsc_continue_ra against the oracle's continuation (Sec. 4.3) on the RW4 branch from
    the same oracle-made estimate: the same Ra sequence and Newton counts, and waves that
    agree to the converged-wave tolerance."""
    from oracle import continuation as ct
    from paper_2508_16635_gb300 import RotatingShell
    L, Ms, Nr, Ek, M = 31, 4, 24, 1e-3, 4
    s = Shell(L, Ms, Nr, Ek, 120.0)
    U0, C0, J = _rw_initial_guess(s, M)
    kw = dict(n_opt=4, gamma=20.0, max_points=4, kmax=150)
    pts_o = ct.continue_ra(s, U0, C0, J, 120.0, 121.0, 200.0, **kw)
    gpu = RotatingShell(L, Ms, Nr, Ek, 120.0)
    U = torch.tensor(U0, device="cuda")
    pts_g, Cg, st = gpu.continue_ra(U, C0, J, 120.0, 121.0, 200.0, **kw)
    assert st == 0 and len(pts_g) == len(pts_o) == 4
    for a, b in zip(pts_o, pts_g):
        assert a["its"] == b["newton_iterations"]
        assert abs(a["Ra"] - b["Ra"]) <= 1e-12 * a["Ra"]
        assert b["residual"] < 1e-10
        assert abs(a["C"] - b["C"]) <= 1e-9 * abs(a["C"])
        ke = s.kinetic_energy(a["U"])
        assert abs(ke - b["KE"]) <= 1e-8 * ke
    assert _rel(U.cpu().numpy(), pts_o[-1]["U"]) < 1e-9
    assert Cg == pts_g[-1]["C"]
    gpu.close()


def test_batch_jacobian_parity(torch):
    """rsc_batch_apply_jacobian: instances of different symmetries and Ra in one graph launch,
    each against the oracle's Jacobian action; a second call with new directions in the same
    buffers replays the graph."""
    from paper_2508_16635_gb300 import Batch
    inst = [dict(L=15, Ms=4, Nr=12, Ek=1e-3, Ra=100.0), dict(L=15, Ms=6, Nr=12, Ek=1e-3, Ra=130.0),
            dict(L=13, Ms=3, Nr=11, Ek=3e-3, Ra=90.0)]
    b = Batch(inst)
    shells = [Shell(d["L"], d["Ms"], d["Nr"], d["Ek"], d["Ra"]) for d in inst]
    count, dt, C = 2, 200.0, [0.3, -0.7, 1.1]
    J = [shells[0].real_index("T", 4, 4, 1, 1), None, shells[2].real_index("T", 3, 3, 2, 1)]
    U = [s.conductive_state() + si.perturbation(s.L, s.Ms, s.Nr, seed=50 + i, amp=3e-2)
         for i, s in enumerate(shells)]
    Ug = [torch.tensor(x, device="cuda") for x in U]
    ug = [torch.zeros(count * s.n, dtype=torch.float64, device="cuda") for s in shells]
    out = [torch.zeros_like(x) for x in ug]
    for rep in range(2):
        dirs = []
        for i, s in enumerate(shells):
            d = np.concatenate([si.random_vector(s.L, s.Ms, s.Nr, seed=100 * rep + 10 * i + q)
                                for q in range(count)])
            if J[i] is not None:
                d[J[i]] = 0.4
                d[s.n + J[i]] = -0.2
            dirs.append(d)
            ug[i].copy_(torch.tensor(d, device="cuda"))
        b.apply_jacobian(Ug, C, J, ug, dt, out=out)
        b.synchronize()
        for i, s in enumerate(shells):
            got = out[i].cpu().numpy()
            for q in range(count):
                want = s.jvp(U[i], C[i], J[i], dirs[i][q * s.n:(q + 1) * s.n], dt)
                assert _rel(got[q * s.n:(q + 1) * s.n], want) < 1e-9
    b.close()


def test_batch_instances_share_factorisations(torch):
    """Instances with the same operator (here three Rayleigh numbers at one Ek) share one
    factorisation per dt, an instance at another Ek has its own: every instance's Jacobian
    actions equal those of a lone context bit for bit, and the shared batch holds less
    device memory than the same instances with separate factorisations."""
    from paper_2508_16635_gb300 import Batch, RotatingShell
    L, Ms, Nr = 31, 4, 24
    inst = [dict(L=L, Ms=Ms, Nr=Nr, Ek=1e-3, Ra=Ra) for Ra in (100.0, 120.0, 140.0)]
    inst.append(dict(L=L, Ms=Ms, Nr=Nr, Ek=2e-3, Ra=120.0))
    s = _shell(L, Ms, Nr, 1e-3, 100.0)
    U = [torch.tensor(s.conductive_state() + si.perturbation(L, Ms, Nr, seed=80 + i, amp=3e-2),
                      device="cuda") for i in range(len(inst))]
    u = [torch.tensor(si.random_vector(L, Ms, Nr, seed=90 + i), device="cuda")
         for i in range(len(inst))]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    b = Batch(inst)
    out = [torch.empty_like(x) for x in u]
    b.apply_jacobian(U, [0.3] * 4, [None] * 4, u, 200.0, out=out)
    b.synchronize()
    used_shared = free0 - torch.cuda.mem_get_info()[0]
    for i, d in enumerate(inst):
        lone = RotatingShell(L, Ms, Nr, d["Ek"], d["Ra"])
        ref = lone.apply_jacobian(U[i], 0.3, None, u[i], 200.0)
        assert torch.equal(ref, out[i]), i
        lone.close()
    b.close()
    torch.cuda.synchronize()
    # the same four instances as lone contexts (four factorisations instead of two)
    free1 = torch.cuda.mem_get_info()[0]
    lones = [RotatingShell(L, Ms, Nr, d["Ek"], d["Ra"]) for d in inst]
    for i, g in enumerate(lones):
        g.apply_jacobian(U[i], 0.3, None, u[i], 200.0)
    torch.cuda.synchronize()
    used_lone = free1 - torch.cuda.mem_get_info()[0]
    for g in lones:
        g.close()
    assert used_shared < used_lone, (used_shared, used_lone)


def test_batch_newton_matches_single_instance_solves(torch):
    """rsc_batch_newton_rw (instances concurrently) gives bit-identical waves to the
    single-context solves (whose parity with the oracle is tested above)."""
    from paper_2508_16635_gb300 import Batch, RotatingShell
    L, Ms, Nr, Ek, M = 31, 4, 24, 1e-3, 4
    s = Shell(L, Ms, Nr, Ek, 120.0)
    U0, C0, J = _rw_initial_guess(s, M)
    inst = [dict(L=L, Ms=Ms, Nr=Nr, Ek=Ek, Ra=Ra) for Ra in (120.0, 121.0)]
    b = Batch(inst)
    Ub = [torch.tensor(U0, device="cuda") for _ in inst]
    Cb, reps, sts = b.newton_rw(Ub, [C0, C0], [J, J], tol=1e-10, max_newton=10, kmax=150)
    assert sts == [0, 0]
    for i, d in enumerate(inst):
        g = RotatingShell(L, Ms, Nr, Ek, d["Ra"])
        Us = torch.tensor(U0, device="cuda")
        Cs, rep, st = g.newton_rw(Us, C0, J, tol=1e-10, max_newton=10, kmax=150)
        assert st == 0 and Cs == Cb[i] and torch.equal(Us, Ub[i])
        assert rep["iterations"] == reps[i]["iterations"]
        g.close()
    b.close()


@pytest.mark.parametrize("name,L,Ms,Nr,Ek,Ra", CASES_C3)
@pytest.mark.parametrize("cluster", [16, 8, 4, 2])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_chain_sweep_variants_parity(torch, name, L, Ms, Nr, Ek, Ra, cluster, mode):
    """Every FP64 sweep variant the tuner can pick (chain_async 0: cluster barrier per block;
    1 / 2: two / four warps per row group with st.async / mbarrier exchange) on every
    cluster size the device schedules, against the oracle: a step at dt = 2e-3 and a
    Jacobian action with the drift unknown at dt = 200, both at the FP64 bound."""
    from paper_2508_16635_gb300 import RotatingShell
    s = _shell(L, Ms, Nr, Ek, Ra)
    x, want = _oracle_step(L, Ms, Nr, Ek, Ra, 22, 1e-2, -2.7, 2e-3, 2)
    U0, u, J, wantj = _oracle_jvp(L, Ms, Nr, Ek, Ra, 23, True, -1.1, 200.0)
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra)
    t = gpu.tuning()
    t.update(chain_cluster=cluster, chain_async=mode)
    try:
        gpu.set_tuning(t)
    except Exception:
        gpu.close()
        pytest.skip(f"cluster of {cluster} not schedulable for N_r = {Nr}")
    U = torch.tensor(x, device="cuda")
    gpu.step(U, -2.7, 2e-3, nsteps=2)
    errs = _maxabs_fields(s, U.cpu().numpy(), want)
    assert max(errs) < 1e-11, errs
    got = gpu.apply_jacobian(torch.tensor(U0, device="cuda"), -1.1, J,
                             torch.tensor(u, device="cuda"), 200.0).cpu().numpy()
    errs = _maxabs_fields(s, got, wantj)
    assert max(errs) < 1e-11, errs
    gpu.close()


@pytest.mark.parametrize("name,L,Ms,Nr,Ek,Ra", CASES)
def test_autotune_keeps_results_bitwise(torch, name, L, Ms, Nr, Ek, Ra):
    """The autotuner only changes launch shapes (which rows, radii or pairs a block takes),
    never the order of any sum: with the sweep variant held fixed, steps and Jacobian
    actions are bit-identical after it."""
    from paper_2508_16635_gb300 import RotatingShell
    s = Shell(L, Ms, Nr, Ek, Ra)
    x = s.conductive_state() + si.perturbation(L, Ms, Nr, seed=61, amp=3e-2)
    u = si.random_vector(L, Ms, Nr, seed=62)
    for prec in ("fp64", "mixed"):
        gpu = RotatingShell(L, Ms, Nr, Ek, Ra, precision=prec)
        U = torch.tensor(x, device="cuda")
        a0 = gpu.apply_jacobian(U, 0.3, None, torch.tensor(u, device="cuda"), 200.0).clone()
        s0 = gpu.step(U.clone(), 0.0, 1e-3).clone()
        t0 = gpu.tuning()
        t = gpu.autotune()
        assert t["chain_cluster"] in (2, 4, 8, 16) and min(t["rhs_pairs"]) >= 1
        # the sweep variant, the tensor-core analysis and the double-float sweeps' column
        # split sum in another order (the double-float cluster size does not)
        gpu.set_tuning(dict(t, chain_async=0, analysis_tc=0, chain_df=t0["chain_df"],
                            chain_cr=t0["chain_cr"]))
        a1 = gpu.apply_jacobian(U, 0.3, None, torch.tensor(u, device="cuda"), 200.0)
        s1 = gpu.step(U.clone(), 0.0, 1e-3)
        assert torch.equal(a0, a1) and torch.equal(s0, s1)
        bad = dict(t, rhs_pairs=[3, 3])
        with pytest.raises(Exception):
            gpu.set_tuning(bad)
        gpu.close()


def test_regrid_and_spectral_tail_parity(torch):
    """rsc_regrid against the oracle's zero fill (bitwise), both ways; rsc_spectral_tail
    against the ratios computed from the coefficients in numpy."""
    from oracle import continuation as ct
    from paper_2508_16635_gb300 import RotatingShell
    L0, Ms, Nr0, L1, Nr1 = 15, 4, 12, 19, 15
    a = RotatingShell(L0, Ms, Nr0, 1e-3, 100.0)
    b = RotatingShell(L1, Ms, Nr1, 1e-3, 100.0)
    s0 = Shell(L0, Ms, Nr0, 1e-3, 100.0)
    x = s0.conductive_state() + si.perturbation(L0, Ms, Nr0, seed=71)
    Ub = b.regrid_from(a, torch.tensor(x, device="cuda"))
    y = ct.regrid(x, L0, Ms, Nr0, L1, Nr1)
    assert np.array_equal(Ub.cpu().numpy(), y)
    Ua = a.regrid_from(b, Ub)
    assert np.array_equal(Ua.cpu().numpy(), x)
    cheb, sh = a.spectral_tail(torch.tensor(x, device="cuda"))
    z = s0.to_complex(x - s0.conductive_state())
    A = np.abs(z).max()
    assert abs(cheb - np.abs(z[:, :, -1]).max() / A) < 1e-14
    assert abs(sh - np.abs(z[:, s0.pair_l == L0, :]).max() / A) < 1e-14
    a.close()
    b.close()


def test_ek_continuation_parity(torch):
    """rsc_continue_ek against the oracle's continuation in log10 Ek (Sec. 4.4) on the RW4
    branch with Ra = 12 Ek^(-1/3) (Ra = 120 at Ek = 1e-3)."""
    from oracle import continuation as ct
    from paper_2508_16635_gb300 import RotatingShell
    L, Ms, Nr, Ek, M = 31, 4, 24, 1e-3, 4
    s = Shell(L, Ms, Nr, Ek, 120.0)
    U0, C0, J = _rw_initial_guess(s, M)
    kw = dict(n_opt=3, gamma=400.0, max_points=3, kmax=150)
    pts_o = ct.continue_ek(s, U0, C0, J, 1e-3, 0.97e-3, 0.5e-3, ra_coef=12.0, **kw)
    gpu = RotatingShell(L, Ms, Nr, Ek, 120.0)
    U = torch.tensor(U0, device="cuda")
    pts_g, Cg, st = gpu.continue_ek(U, C0, J, 1e-3, 0.97e-3, 0.5e-3, ra_coef=12.0, **kw)
    assert st == 0 and len(pts_g) == len(pts_o) == 3
    for a, b in zip(pts_o, pts_g):
        assert a["its"] == b["newton_iterations"]
        assert abs(10 ** a["Ra"] - b["Ek"]) <= 1e-12 * b["Ek"]
        assert abs(b["Ra"] - 12.0 * b["Ek"] ** (-1.0 / 3.0)) < 1e-10
        assert b["residual"] < 1e-10
        assert abs(a["C"] - b["C"]) <= 1e-9 * abs(a["C"])
    assert _rel(U.cpu().numpy(), pts_o[-1]["U"]) < 1e-9
    gpu.close()


def test_ek_continuation_refines_the_grid(torch):
    """A tail threshold below the wave's own tail forces one refinement: the continuation
    resumes on the finer grid from the regridded wave, which converges to nearly the same
    drift (the coarse grid already resolves it to about 1e-4)."""
    from paper_2508_16635_gb300.rsc import RotatingShell, follow_ek
    L, Ms, Nr, Ek, M = 31, 4, 24, 1e-3, 4
    s = Shell(L, Ms, Nr, Ek, 120.0)
    U0, C0, J = _rw_initial_guess(s, M)
    k_phase = (J // 2) % Nr
    gpu = RotatingShell(L, Ms, Nr, Ek, 120.0)
    U = torch.tensor(U0, device="cuda")
    cheb, sh = gpu.spectral_tail(U)
    thr = 0.5 * max(cheb, sh)
    pts, fine, Uf, Cf = follow_ek(gpu, U, C0, M, k_phase, 1e-3, 0.98e-3, 0.9e-3, tail_threshold=thr,
                                  max_refinements=1, ra_coef=12.0, max_points=3, kmax=150)
    assert (fine.L, fine.Nr) != (L, Nr)
    coarse = [p for p in pts if (p["L"], p["Nr"]) == (L, Nr)]
    refined = [p for p in pts if (p["L"], p["Nr"]) == (fine.L, fine.Nr)]
    assert coarse and refined and refined[0]["residual"] < 1e-10
    assert abs(refined[0]["Ek"] - coarse[-1]["Ek"]) < 1e-15
    assert abs(refined[0]["C"] - coarse[-1]["C"]) < 1e-3 * abs(coarse[-1]["C"])
    fine.close()
    gpu.close()


# ---- the implicit solve on its own (Sec. 3.2): backward error against the oracle's chains ---
def _random_rhs(s, seed):
    """Random right-hand side at the collocation radii: real at m = 0, zero in the rows of
    e_00 and f_00 (the structure of every right-hand side the library forms)."""
    rng = np.random.default_rng(seed)
    b = rng.standard_normal((3, s.P, s.Nr)) + 1j * rng.standard_normal((3, s.P, s.Nr))
    b[:, s.pair_m == 0] = b[:, s.pair_m == 0].real
    b[:2, s.pair_l == 0] = 0.0
    return b


def _solve_errors(s, dt, b, x):
    """(worst row-scaled backward error of the e/f chains in the oracle's assembled system,
    max_i |A x - b|_i / (||A_i||_1 ||x_chain||_inf + |b_i|); worst max-abs difference of a
    chain's solution from the oracle's solve over its largest entry; the same for T)."""
    xo = s.solve(b, dt)
    worst_eta = worst_fwd = 0.0
    for a, m in enumerate(s.ms):
        p0 = s.starts[a]
        for cls in (0, 1):
            flds, D, A, C = s.chain_system(m, cls, dt)
            fi = [0 if f == "e" else 1 for f in flds]
            xs = [x[fi[i], p0 + i] for i in range(len(D))]
            bs = [b[fi[i], p0 + i] for i in range(len(D))]
            xn = max(float(np.abs(v).max()) for v in xs)
            for i in range(len(D)):
                r = D[i] @ xs[i] - bs[i]
                rown = np.abs(D[i]).sum(axis=1)
                if A[i] is not None:
                    r = r + A[i] @ xs[i - 1]
                    rown = rown + np.abs(A[i]).sum(axis=1)
                if C[i] is not None:
                    r = r + C[i] @ xs[i + 1]
                    rown = rown + np.abs(C[i]).sum(axis=1)
                worst_eta = max(worst_eta, float((np.abs(r) / (rown * xn + np.abs(bs[i]))).max()))
            xo_c = np.concatenate([xo[fi[i], p0 + i] for i in range(len(D))])
            worst_fwd = max(worst_fwd, float(np.abs(xo_c - np.concatenate(xs)).max()
                                             / np.abs(xo_c).max()))
    fwd_T = float(np.abs(xo[2] - x[2]).max() / np.abs(xo[2]).max())
    return worst_eta, worst_fwd, fwd_T


@pytest.mark.parametrize("name,L,Ms,Nr,Ek,Ra", CASES_C3)
@pytest.mark.parametrize("dt", [2e-3, 200.0])
def test_implicit_solve_backward_error_fp64(torch, name, L, Ms, Nr, Ek, Ra, dt):
    """rsc_implicit_solve with every FP64 sweep variant and cluster size the device schedules:
    row-scaled backward error in the oracle's assembled chains below 64 u, and the solution
    within 1e-11 of the oracle's (temperature 1e-12)."""
    from paper_2508_16635_gb300 import RotatingShell
    s = _shell(L, Ms, Nr, Ek, Ra)
    b = _random_rhs(s, 90 + L)
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra)
    t0 = gpu.tuning()
    B = torch.tensor(s.to_real(b), device="cuda")
    ran = 0
    for mode in (0, 1, 2):
        for cs in (16, 8, 4, 2):
            try:
                gpu.set_tuning(dict(t0, chain_cluster=cs, chain_async=mode))
            except Exception:
                continue
            ran += 1
            x = s.to_complex(gpu.implicit_solve(B, dt).cpu().numpy())
            eta, fwd, fwd_T = _solve_errors(s, dt, b, x)
            assert eta < 64 * U64, (mode, cs, eta / U64)
            assert fwd < 1e-11, (mode, cs, fwd)
            assert fwd_T < 1e-12, (mode, cs, fwd_T)
    assert ran >= 3
    gpu.close()


def _longest_chain(L):
    return L + 1       # blocks of the m = 0 chains (one per degree l, e and f alternating)


@pytest.mark.parametrize("name,L,Ms,Nr,Ek,Ra", CASES_C3)
@pytest.mark.parametrize("dt", [2e-3, 200.0])
def test_implicit_solve_backward_error_double_float(torch, name, L, Ms, Nr, Ek, Ra, dt):
    """The double-float chain solve of the mixed path (chain_df = 2 / 4, every schedulable
    cluster size, and chains cut into 2 and 4 parts where a chain has enough blocks) on its
    own, against the oracle's chains: the tables carry 2^-48 relative (FP32 hi + lo), so the
    row-scaled backward error stays below 64 u_df and the solution within 32 x the FP64
    bound.  The partitioned solves must run their spike kernels (more launches)."""
    from paper_2508_16635_gb300 import RotatingShell
    s = _shell(L, Ms, Nr, Ek, Ra)
    b = _random_rhs(s, 95 + L)
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra, precision="mixed")
    t0 = gpu.tuning()
    assert t0["chain_df"] in (2, 4) and t0["chain_cr"] == 1   # the defaults of a mixed context
    B = torch.tensor(s.to_real(b), device="cuda")
    ran = 0
    for ns in (2, 4):
        for cs in (16, 8, 4, 2):
            try:
                gpu.set_tuning(dict(t0, chain_df=ns, chain_df_cluster=cs, chain_parts=1,
                                    chain_cr=0))
            except Exception:
                continue
            ran += 1
            x = s.to_complex(gpu.implicit_solve(B, dt).cpu().numpy())
            eta, fwd, fwd_T = _solve_errors(s, dt, b, x)
            assert eta < 64 * U48, (ns, cs, eta / U48)
            assert fwd < 32 * 1e-11, (ns, cs, fwd)
            assert fwd_T < 1e-12, (ns, cs, fwd_T)
    assert ran >= 2
    # partitioned chains (SPIKE-type): only where the longest chain splits into parts of at
    # least 8 blocks; a failing set_tuning is an error here
    for parts in (2, 4):
        if _longest_chain(L) < 8 * parts:
            continue
        gpu.set_tuning(dict(t0, chain_parts=1, chain_cr=0))
        gpu.implicit_solve(B, dt)
        torch.cuda.synchronize()
        n1 = gpu.launch_count()
        gpu.implicit_solve(B, dt)
        torch.cuda.synchronize()
        plain = gpu.launch_count() - n1
        gpu.set_tuning(dict(t0, chain_parts=parts))
        gpu.implicit_solve(B, dt)       # refactorises
        torch.cuda.synchronize()
        n1 = gpu.launch_count()
        x = s.to_complex(gpu.implicit_solve(B, dt).cpu().numpy())
        torch.cuda.synchronize()
        assert gpu.launch_count() - n1 > plain, "the spike kernels did not run"
        eta, fwd, fwd_T = _solve_errors(s, dt, b, x)
        assert eta < 64 * U48, (parts, eta / U48)
        assert fwd < 32 * 1e-11, (parts, fwd)
    gpu.close()


@pytest.mark.parametrize("name,L,Ms,Nr,Ek,Ra", CASES_C3)
@pytest.mark.parametrize("dt", [2e-3, 200.0])
def test_implicit_solve_backward_error_reduced_chains(torch, name, L, Ms, Nr, Ek, Ra, dt):
    """The double-float solve on odd-even reduced chains (chain_cr = 1: the odd blocks
    eliminated with D_i^-1, the half-length chains of the even blocks swept, the odd blocks
    recovered from their neighbours) with 2 / 4 warps per row group on every schedulable
    cluster size, against the oracle's chains: row-scaled backward error below 64 u_df, the
    solution within 32 x the FP64 bound of the reduced factors on the host (1e-10 at L = 127,
    N_r = 64, dt = 200, where the odd blocks' back-substitution cancels O(1) Coriolis terms
    against an O(Ek) diagonal; tests/test_host_factor_cr.py).  The reduced passes must run:
    two launches more than the unreduced solve."""
    from paper_2508_16635_gb300 import RotatingShell
    s = _shell(L, Ms, Nr, Ek, Ra)
    b = _random_rhs(s, 97 + L)
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra, precision="mixed")
    t0 = gpu.tuning()
    B = torch.tensor(s.to_real(b), device="cuda")

    def launches(**kw):
        gpu.set_tuning(dict(t0, **kw))
        gpu.implicit_solve(B, dt)
        torch.cuda.synchronize()
        n1 = gpu.launch_count()
        x = gpu.implicit_solve(B, dt).cpu().numpy()
        torch.cuda.synchronize()
        return gpu.launch_count() - n1, x

    plain, _ = launches(chain_df=2, chain_cr=0)
    ran = 0
    for ns in (2, 4):
        for cs in (16, 8, 4, 2):
            try:
                gpu.set_tuning(dict(t0, chain_df=ns, chain_df_cluster=cs, chain_cr=1))
            except Exception:
                continue
            ran += 1
            n, x = launches(chain_df=ns, chain_df_cluster=cs, chain_cr=1)
            assert n == plain + 2, (ns, cs, n, plain)
            eta, fwd, fwd_T = _solve_errors(s, dt, b, s.to_complex(x))
            assert eta < 64 * U48, (ns, cs, eta / U48)
            assert fwd < 32 * 1e-10, (ns, cs, fwd)
            assert fwd_T < 1e-12, (ns, cs, fwd_T)
    assert ran >= 2
    gpu.close()


@pytest.mark.parametrize("name,L,Ms,Nr,Ek,Ra", CASES_C3)
@pytest.mark.parametrize("dt", [2e-3, 200.0])
def test_gpu_reduced_factorisation_matches_the_host(torch, name, L, Ms, Nr, Ek, Ra, dt):
    """The factorisation of the odd-even reduced chains on the GPU (factor_gpu = 1: FP64
    block LU of the odd blocks, the reduced blocks from the Chebyshev tables, the twisted
    factors of the reduced chains) against the host routine (factor_gpu = 0, pinned by
    tests/test_host_factor_cr.py), block by block: D_i^-1 of every odd block and G', H', W'
    of every reduced block, within 1e-9 of each block's largest entry (the blocks'
    condition numbers reach 1e6 at L = 127, N_r = 64); both then pass the backward-error
    check of the reduced double-float solve."""
    from paper_2508_16635_gb300 import RotatingShell
    s = _shell(L, Ms, Nr, Ek, Ra)
    ctxs = []
    for flag in (1, 0):
        c = RotatingShell(L, Ms, Nr, Ek, Ra, precision="mixed")
        c.set_tuning(dict(c.tuning(), factor_gpu=flag, chain_cr=1))
        ctxs.append(c)
    gpu, host = ctxs
    nodd = sum(2 * ((L - m + 1) // 2) for m in s.ms)
    nred = 2 * s.P - nodd
    worst = {}
    for w, n in (("Dinv", nodd), ("Gr", nred), ("Hr", nred), ("Wr", nred)):
        worst[w] = 0.0
        for b in range(n):
            a, h = gpu.factor_block(dt, w, b), host.factor_block(dt, w, b)
            scale = np.abs(h).max()
            if scale == 0.0:
                assert np.abs(a).max() == 0.0, (w, b)
                continue
            worst[w] = max(worst[w], float(np.abs(a - h).max() / scale))
    assert gpu.factor_time_cr()[1] and not host.factor_time_cr()[1]
    assert max(worst.values()) < 1e-9, worst
    b = _random_rhs(s, 98 + L)
    B = torch.tensor(s.to_real(b), device="cuda")
    for ctx in (gpu, host):
        x = s.to_complex(ctx.implicit_solve(B, dt).cpu().numpy())
        eta, fwd, fwd_T = _solve_errors(s, dt, b, x)
        assert eta < 64 * U48 and fwd < 32 * 1e-10 and fwd_T < 1e-12, (eta / U48, fwd, fwd_T)
    gpu.close()
    host.close()


@pytest.mark.parametrize("name,L,Ms,Nr,Ek,Ra", CASES_C3)
@pytest.mark.parametrize("dt", [2e-3, 200.0])
def test_gpu_factorisation_matches_the_host_factors(torch, name, L, Ms, Nr, Ek, Ra, dt):
    """The FP64 block factorisation on the GPU (factor_gpu = 1, the default) against the
    host routine (factor_gpu = 0), block by block: G, H, W of every chain block and the
    temperature inverses.  The two sum in different orders; the factors' sensitivity to
    rounding is the condition number of the equilibrated blocks D' (up to about 1e6 at
    L = 127, N_r = 64), so blocks agree to 1e-9 of their largest entry and the temperature
    inverses (condition about 1e4) to 1e-11; both factorisations then pass the solve's
    backward-error check."""
    from paper_2508_16635_gb300 import RotatingShell
    s = _shell(L, Ms, Nr, Ek, Ra)
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra)
    host = RotatingShell(L, Ms, Nr, Ek, Ra)
    host.set_tuning(dict(host.tuning(), factor_gpu=0))
    assert gpu.tuning()["factor_gpu"] == 1
    nblk = 2 * s.P
    worst = {"G": 0.0, "H": 0.0, "W": 0.0}
    for b in range(nblk):
        for w in ("G", "H", "W"):
            a, h = gpu.factor_block(dt, w, b), host.factor_block(dt, w, b)
            scale = np.abs(h).max()
            if scale == 0.0:
                assert np.abs(a).max() == 0.0, (w, b)
                continue
            worst[w] = max(worst[w], float(np.abs(a - h).max() / scale))
    assert gpu.factor_time()[1] and not host.factor_time()[1]
    assert max(worst.values()) < 1e-9, worst
    for l in range(L + 1):
        a, h = gpu.factor_block(dt, "T", l), host.factor_block(dt, "T", l)
        assert np.abs(a - h).max() < 1e-11 * np.abs(h).max(), l
    b = _random_rhs(s, 99 + L)
    for ctx in (gpu, host):
        x = s.to_complex(ctx.implicit_solve(torch.tensor(s.to_real(b), device="cuda"), dt)
                         .cpu().numpy())
        eta, fwd, fwd_T = _solve_errors(s, dt, b, x)
        assert eta < 64 * U64 and fwd < 1e-11 and fwd_T < 1e-12, (eta / U64, fwd, fwd_T)
    gpu.close()
    host.close()


@pytest.mark.parametrize("name,L,Ms,Nr,Ek,Ra", CASES_C3)
@pytest.mark.parametrize("chain_cr", [0, 1])
def test_double_float_chain_solve_against_the_oracle(torch, name, L, Ms, Nr, Ek, Ra, chain_cr):
    """The mixed Jacobian action with the double-float chain solve (unreduced and odd-even
    reduced chains) against the FP64 oracle, at the mixed-path bound (the FP32 transforms
    dominate): 5e-5 per field."""
    from paper_2508_16635_gb300 import RotatingShell
    s = _shell(L, Ms, Nr, Ek, Ra)
    x = s.conductive_state() + si.perturbation(L, Ms, Nr, seed=73, amp=1e-2)
    u = si.random_vector(L, Ms, Nr, seed=74)
    J = s.real_index("T", Ms, Ms, 1, 1)
    want = s.jvp(x, 0.4, J, u, 200.0)
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra, precision="mixed")
    assert gpu.tuning()["chain_df"] in (2, 4)
    gpu.set_tuning(dict(gpu.tuning(), chain_cr=chain_cr))
    got = gpu.apply_jacobian(torch.tensor(x, device="cuda"), 0.4, J,
                             torch.tensor(u, device="cuda"), 200.0).cpu().numpy()
    errs = _maxabs_fields(s, got, want)
    assert max(errs) < 5e-5, errs
    gpu.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_krylov_split_basis_newton_matches_fp64_basis(torch, precision):
    """GMRES with the double-float copy of the Krylov basis (krylov_split = 1, the default)
    against the FP64 passes (krylov_split = 0) on the RW4 solve: both converge to 1e-11 and
    reach the same wave (state and drift within 1e-10 relative)."""
    from paper_2508_16635_gb300 import RotatingShell
    L, Ms, Nr, Ek, Ra = 23, 4, 20, 1e-3, 120.0
    s = Shell(L, Ms, Nr, Ek, Ra)
    U0, C0, J = _rw_initial_guess(s, 4)
    out = {}
    for split in (1, 0):
        gpu = RotatingShell(L, Ms, Nr, Ek, Ra, precision=precision)
        assert gpu.tuning()["krylov_split"] == 1
        gpu.set_tuning(dict(gpu.tuning(), krylov_split=split))
        U = torch.tensor(U0, device="cuda")
        C, rep, st = gpu.newton_rw(U, C0, J, tol=1e-11, max_newton=14, kmax=120, gmres_tol=1e-10)
        assert st == 0, rep
        out[split] = (U.cpu().numpy(), C, rep)
        gpu.close()
    (U1, C1, r1), (U0_, C0_, r0) = out[1], out[0]
    assert _rel(U1, U0_) < 1e-10
    assert abs(C1 - C0_) < 1e-10 * abs(C0_)
    assert abs(r1["iterations"] - r0["iterations"]) <= 1


# ---- the RW12 wave at the benchmark truncation against the oracle's (Table 1 row 3) -------
def _golden_rw12():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rw12_c3_oracle.txt")
    vals = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def _gpu_rw12_guess(torch, RotatingShell, L, Ms, Nr, Ek, Ra, M):
    """The oracle's route to the wave on the GPU: the same m = 12 seed, IMEX Euler steps of
    dt = 1e-4 until the m = 12 temperature amplitude settles (the recipe of
    tests/golden/make_rw12_c3.py), drift from the phase rate, slot J of Sec. 3.4."""
    import cmath
    sh = RotatingShell(L, Ms, Nr, Ek, Ra)
    U = sh.conductive_state() + torch.tensor(si.mode_seed(L, Ms, Nr, M, seed=4000, amp=1e-2),
                                             device="cuda")
    x = U.view(3, sh.P, Nr, 2)
    pM = L + 1
    prev, steps = None, 0
    while steps < 6000:
        sh.step(U, 0.0, 1e-4, nsteps=100)
        steps += 100
        amp = float(torch.linalg.norm(x[2, pM]).item())
        if prev is not None and amp > 1e-3 and abs(amp - prev) < 1e-4 * amp:
            break
        prev = amp
    a0 = x[2, pM].clone()
    sh.step(U, 0.0, 1e-4, nsteps=10)
    a1 = x[2, pM]
    k = int(torch.argmax(a0[:, 0] ** 2 + a0[:, 1] ** 2).item())
    C0 = -cmath.phase(complex(a1[k, 0].item(), a1[k, 1].item()) /
                      complex(a0[k, 0].item(), a0[k, 1].item())) / (M * 10 * 1e-4)
    kstar = int(torch.argmax(torch.abs(x[2, pM, :, 0])).item())
    J = sh.phase_slot(M, kstar)
    sh.close()
    return U, C0, J


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_rw12_wave_against_the_oracle_wave(torch, precision):
    """Table 1 row 3 parameters (Ek = 1e-5, Ra = 140, M = 12) at L = 127, N_r = 64: the wave
    converged by the GPU's Newton-GMRES (FP64 residual to 1e-10) against the oracle's wave
    (tests/golden/rw12_c3_oracle.txt, written by make_rw12_c3.py from oracle/ only): drift
    speed, kinetic energy and both Nusselt numbers within 1e-8 relative on the FP64 and on
    the mixed path (the target is the drift within 1e-8 of the FP64 oracle)."""
    from paper_2508_16635_gb300 import RotatingShell
    want = _golden_rw12()
    L, Ms, Nr, Ek, Ra, M = 127, 12, 64, 1e-5, 140.0, 12
    U, C0, J = _gpu_rw12_guess(torch, RotatingShell, L, Ms, Nr, Ek, Ra, M)
    gpu = RotatingShell(L, Ms, Nr, Ek, Ra, precision=precision)
    C, rep, st = gpu.newton_rw(U, C0, J, tol=1e-10, max_newton=12, kmax=600, gmres_tol=1e-10)
    assert st == 0 and rep["residual"] < 1e-10, rep
    ke, nu_in, nu_out = gpu.diagnostics(U)
    errs = {"C": abs(C - want["C"]) / abs(want["C"]), "KE": abs(ke - want["KE"]) / want["KE"],
            "Nu_in": abs(nu_in - want["Nu_in"]) / want["Nu_in"],
            "Nu_out": abs(nu_out - want["Nu_out"]) / want["Nu_out"]}
    print(precision, errs)
    assert max(errs.values()) < 1e-8, errs
    gpu.close()


# ---- linear onset (oracle/onset.py; Secs. 2.2, 4.4) ----------------------------------------
def _golden_onset():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "onset_workloads.txt")
    rows = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            rows[f[0]] = dict(Ek=float(f[1]), m=int(f[2]), L=int(f[3]), Nr=int(f[4]),
                              Ra=float(f[5]), omega=float(f[6]), C=float(f[7]))
    return rows


@functools.lru_cache(maxsize=None)
def _onset_mode(name):
    """The oracle's neutral mode of a workload at its stored onset (make_onset.py): Arnoldi
    near i omega on the pencil at Ra_c; (state vector, sigma, row)."""
    from oracle import onset as on
    g = _golden_onset()[name]
    pen = on.Pencil(Shell(g["L"], g["m"], g["Nr"], g["Ek"], 1.0), g["m"], 1)
    sig, V = on.eig_near(pen, g["Ra"], 1j * g["omega"], k=4)
    j = int(np.argmin(np.abs(sig - 1j * g["omega"])))
    return pen.state(V[:, j] / np.linalg.norm(V[:, j])), complex(sig[j]), g


@pytest.mark.parametrize("name", ["C1", "C2"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_linearised_step_fixes_the_onset_mode(torch, name, precision):
    """At the workload's onset (Ra_c) with the onset drift C_c = -omega/m in the explicit
    part, the GPU's linearised step at the conductive state leaves the oracle's neutral mode
    unchanged: |(B_U - I) u| / |u| below 1e-10 in FP64 (below 1e-4 on the mixed path, whose
    FP32 transforms move a Jacobian action by about 2e-5), at the Newton pseudo-timestep and
    at a short one.  Off onset (Ra = 0.9 Ra_c) it does not."""
    from paper_2508_16635_gb300 import RotatingShell
    u, sig, g = _onset_mode(name)
    M = g["m"]
    C = -sig.imag / M
    bound = 1e-10 if precision == "fp64" else 1e-4
    gpu = RotatingShell(g["L"], M, g["Nr"], g["Ek"], g["Ra"], precision=precision)
    U = gpu.conductive_state()
    ut = torch.tensor(u, device="cuda")
    for dt in (200.0, 1e-3):
        r = gpu.apply_jacobian(U, C, None, ut, dt).cpu().numpy()
        assert np.linalg.norm(r) < bound * np.linalg.norm(u), (dt, np.linalg.norm(r))
    gpu.set_params(Ra=0.9 * g["Ra"])
    r = gpu.apply_jacobian(gpu.conductive_state(), C, None, ut, 200.0).cpu().numpy()
    assert np.linalg.norm(r) > 1e-3 * np.linalg.norm(u)
    gpu.close()


def test_rw_branch_meets_the_onset_on_the_gpu(torch):
    """The nonlinear branch against the linear onset: RW4 (Ek = 1e-3) followed down in Ra by
    the GPU's Newton-GMRES from Table 1's Ra = 120 to 1.01 Ra_c.  Near a supercritical onset
    the kinetic energy grows like Ra - Ra_c and the drift tends to the onset drift, so the
    linear extrapolation of KE and C from 1.01 and 1.02 Ra_c gives Ra_c within 5e-4 and C_c
    within 2e-4 of the oracle's pencil (L = 23, N_r = 16; the oracle's own branch lands
    within 1.0e-4 and 2.1e-5)."""
    from oracle import krylov
    from oracle import onset as on
    from paper_2508_16635_gb300 import RotatingShell
    L, Ms, Nr, Ek, M = 23, 4, 16, 1e-3, 4
    lin = on.critical_rayleigh(on.Pencil(Shell(L, M, Nr, Ek, 1.0), M, 1), (40.0, 80.0),
                               shift="auto")
    s = Shell(L, Ms, Nr, Ek, 120.0)
    U0, C0, J = _rw_initial_guess(s, M)
    gpu = RotatingShell(L, Ms, Nr, Ek, 120.0)
    U = torch.tensor(U0, device="cuda")
    Uc = gpu.conductive_state()
    C, rep, st = gpu.newton_rw(U, C0, J, tol=1e-11, max_newton=14, kmax=150)
    assert st == 0, rep
    Ra_prev = 120.0
    pts = []
    for f in (1.6, 1.3, 1.15, 1.07, 1.04, 1.02, 1.01):
        Ra = f * lin["Ra"]
        # weakly nonlinear predictor: the amplitude scales like sqrt(Ra - Ra_c)
        U.copy_(Uc + (U - Uc) * np.sqrt((Ra - lin["Ra"]) / (Ra_prev - lin["Ra"])))
        gpu.set_params(Ra=Ra)
        C, rep, st = gpu.newton_rw(U, C, J, tol=1e-11, max_newton=20, kmax=200)
        assert st == 0 and rep["residual"] < 1e-11, (f, rep)
        pts.append((Ra, gpu.diagnostics(U)[0], C))
        Ra_prev = Ra
    (Ra2, k2, c2), (Ra1, k1, c1) = pts[-2], pts[-1]
    Ra_ext = Ra1 - k1 * (Ra2 - Ra1) / (k2 - k1)
    C_ext = c1 + (c2 - c1) * (Ra_ext - Ra1) / (Ra2 - Ra1)
    print("onset", lin["Ra"], Ra_ext, lin["C"], C_ext)
    assert abs(Ra_ext - lin["Ra"]) < 5e-4 * lin["Ra"]
    assert abs(C_ext - lin["C"]) < 2e-4 * abs(lin["C"])
    gpu.close()
