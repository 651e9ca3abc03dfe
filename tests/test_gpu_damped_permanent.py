"""Thole-damped permanent polarising field (thole_perm = 1, AMOEBA's rule; the paper damps
only the induced dipoles) on the GPU against the oracle's ``damp_permanent`` option, which
test_oracle_damped_permanent.py pins to the two-site closed forms.

  * multipole_field mode 0 (masked, same body) and mode 2 (masked, whole system): FP64
    kernel, relative 1e-12 of the largest entry; mode 1 (energy potentials) stays undamped;
  * Delta G_solv of the FP64 direct solve with the damped permanent field: 1e-10 relative,
    and it differs from the undamped value by far more than that bar;
  * the adjoint gradient refuses thole_perm = 1 with BEMPOL_ERR_ARG.
"""
import numpy as np
import pytest

import gen
from oracle import multipole as mp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import build_library
    build_library()
    import paper_1810_03698_gb300 as mod
    return mod


def _relmax(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300)


def _damped(pr):
    return gen.with_params(pr, gmres_tol=1e-13, scf_tol=1e-12, scf_maxit=400, damp_permanent=True)


@pytest.mark.parametrize("mode,same_body", [(0, True), (2, False)])
def test_field_mode_matches_oracle(bp, mode, same_body):
    pr = _damped(gen.small_bumpy(3, 40, 8.0))
    st, par = pr.sites, pr.params
    s = bp.problem_solver(pr)
    assert s.params.thole_perm == 1
    mu = np.random.default_rng(11).normal(size=(st.n, 3)) * 0.2
    mu_d = torch.as_tensor(mu, dtype=torch.float64, device="cuda").contiguous()
    E = torch.zeros(st.n * 3, dtype=torch.float64, device="cuda")
    s.multipole_field(E, mu=mu_d, mode=mode)
    F = torch.zeros(st.n * 10, dtype=torch.float64, device="cuda")
    s.multipole_field(F, mu=mu_d, mode=1)
    torch.cuda.synchronize()
    _, g, _ = mp.mult_potentials(st.pos, st.q, st.d, st.Q, mu, st.alpha, st.group, st.body, par.eps_in,
                                 par.thole_a, masked=True, same_body_only=same_body, damp_permanent=True)
    _, g0, _ = mp.mult_potentials(st.pos, st.q, st.d, st.Q, mu, st.alpha, st.group, st.body, par.eps_in,
                                  par.thole_a, masked=True, same_body_only=same_body)
    e = E.cpu().numpy().reshape(-1, 3)
    assert _relmax(e, -g) < 1e-12
    assert _relmax(g0, g) > 1e-6  # the damping changes the field at this site spacing
    P, G, H = mp.mult_potentials(st.pos, st.q, st.d, st.Q, mu, st.alpha, st.group, st.body, par.eps_in,
                                 par.thole_a, masked=False, same_body_only=True)
    f = F.cpu().numpy().reshape(-1, 10)
    iu = np.triu_indices(3)
    assert _relmax(f[:, 0], P) < 1e-12
    assert _relmax(f[:, 1:4], G) < 1e-12
    assert _relmax(f[:, 4:], H[:, iu[0], iu[1]]) < 1e-12
    s.close()


@pytest.mark.parametrize("case", ["sphere1280", "bumpy1280"])
def test_solvation_fp64_direct_damped_matches_oracle(bp, case):
    """The sphere's sites are far apart for the Thole width (the damping changes Delta G by
    ~1e-12 there); the bumpy surface's 40 sites are close enough that it shows."""
    base = gen.sphere_r4_1280() if case == "sphere1280" else gen.small_bumpy(3, 40, 8.0)
    pr = _damped(base)
    ref = mp.solvation(pr, direct_polarization=True)
    s = bp.problem_solver(pr, op="fp64_direct", residual_op="fp64_direct")
    out = s.solve(outputs=True)
    s.close()
    assert abs(out["dG_solv_kcal"] - ref.dG_kcal) < 1e-10 * abs(ref.dG_kcal)
    assert abs(out["G_vac"] - ref.G_vac) < 1e-10 * abs(ref.G_vac)
    assert _relmax(out["mu_diss"].reshape(-1, 3), ref.mu_diss) < 1e-9
    assert _relmax(out["mu_vac"].reshape(-1, 3), ref.mu_vac) < 1e-9
    if case == "bumpy1280":
        s0 = bp.problem_solver(pr, op="fp64_direct", residual_op="fp64_direct", thole_perm=0)
        und = s0.solve()["dG_solv_kcal"]
        s0.close()
        assert abs(und - ref.dG_kcal) > 1e-8 * abs(ref.dG_kcal)


def test_gradient_refuses_damped_permanent(bp):
    pr = _damped(gen.sphere_r4_1280())
    s = bp.problem_solver(pr, op="fp64_direct", residual_op="fp64_direct")
    s.solve()
    with pytest.raises(bp.BempolError) as ei:
        s.gradient()
    assert bp.STATUS[ei.value.status] == "ERR_ARG"
    s.close()
