"""GPU parity of several bodies and several systems in one context.

* A complex AB (two bodies, one solvent) loaded as one system: geometry and the
  near table bit for bit, the matrix-vector product, right-hand side and reaction
  field element by element against the oracle's per-body operators, Delta G_solv
  of the FP64 direct solve within 1e-10 relative.
* The binding triple (A, B, AB) as three systems of one context: each system's
  Delta G_solv equals the oracle's for that problem alone (FP64 direct: 1e-10;
  FP32 treecode with FP64 refinement: 1e-4 relative at theta 0.5, order 5), so
  Delta Delta G_bind = Delta G_AB - Delta G_A - Delta G_B follows.
* Uneven systems (1,280 to 10,240 panels) batched: each system's result equals
  the same system solved in a context of its own.
* Validation of bodies and systems (host-side errors only).
"""
import numpy as np
import pytest

import gen
from oracle import bem, multipole as mp

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


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _relmax(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.fixture(scope="module")
def triple():
    # bodies of subdivision 3 (1,280 panels each), 1 A apart: closer than the near
    # radius 2 sqrt(A) of their panels, so near pairs cross between the bodies
    # tight tolerances on both sides, so the FP64 GPU solve sits on the oracle's exact one
    a, b, ab = (gen.with_params(p, gmres_tol=1e-12, scf_tol=1e-12, scf_maxit=400)
                for p in gen.small_triple(seed_index=411, subdiv=3, radius=7.0, n_sites=16, gap=1.0))
    refs = [mp.solvation(p) for p in (a, b, ab)]
    return (a, b, ab), refs


@pytest.fixture(scope="module")
def complex_ctx(bp, triple):
    (_, _, ab), _ = triple
    par = ab.params
    mesh = bem.build_mesh(ab.verts, ab.tris, par.gauss_k, par.near_factor, body=ab.panel_body)
    s = bp.problem_solver(ab)
    return ab, mesh, s


def test_complex_geometry_and_near_table(complex_ctx):
    ab, mesh, s = complex_ctx
    assert s.systems() == (1, 2)
    g = s.geometry()
    assert np.array_equal(g["centroid"], mesh.cen)
    assert np.array_equal(g["near_ptr"], mesh.near_ptr)
    assert np.array_equal(g["near_col"], mesh.near_cols)
    ref = np.stack(bem.near_correction(mesh, ab.params.kappa), axis=1)
    for k in range(4):
        assert _relmax(g["near_corr"][:, k], ref[:, k]) < 1e-12, k
    rows = np.repeat(np.arange(mesh.n), np.diff(mesh.near_ptr))
    cross = ab.panel_body[rows] != ab.panel_body[mesh.near_cols]
    # near pairs across the bodies carry Yukawa corrections only
    assert cross.any() and not g["near_corr"][cross, :2].any() and g["near_corr"][cross, 2:].any()


@pytest.mark.parametrize("op,bar", [("fp64_direct", 1e-12), ("fp32_direct", 2e-5)])
def test_complex_matvec(complex_ctx, op, bar):
    ab, mesh, s = complex_ctx
    par = ab.params
    A = bem.system_matrix(bem.assemble_layers(mesh, par.kappa), par.eps_in, par.eps_out)
    x = np.random.default_rng(21).normal(size=2 * mesh.n)
    y = torch.zeros(2 * mesh.n, dtype=torch.float64, device="cuda")
    s.matvec(_dev(x), y, op=op)
    assert _relmax(y.cpu().numpy(), A @ x) < bar


def test_complex_rhs_and_reaction(complex_ctx):
    ab, mesh, s = complex_ctx
    st, par = ab.sites, ab.params
    b = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
    s.rhs(b)
    ref = mp.rhs(mesh.cen, st.pos, st.q, st.d, st.Q, par.eps_in, point_body=mesh.body, site_body=st.body)
    assert _relmax(b.cpu().numpy(), ref) < 1e-12
    x = np.random.default_rng(22).normal(size=2 * mesh.n)
    out = torch.zeros(st.n * 10, dtype=torch.float64, device="cuda")
    s.site_reaction(_dev(x), out)
    p, g, h = mp.reaction_at_sites(mesh, x[:mesh.n], x[mesh.n:], st.pos, site_body=st.body)
    o = out.cpu().numpy().reshape(-1, 10)
    assert _relmax(o[:, 0], p) < 1e-12
    assert _relmax(o[:, 1:4], g) < 1e-12
    hh = h[:, [0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]]
    assert _relmax(o[:, 4:], hh) < 1e-12


def test_complex_multipole_modes(complex_ctx):
    ab, mesh, s = complex_ctx
    st, par = ab.sites, ab.params
    mu = np.random.default_rng(23).normal(scale=0.1, size=(st.n, 3))
    for mode, same in ((1, True), (3, False)):
        out = torch.zeros(st.n * 10, dtype=torch.float64, device="cuda")
        s.multipole_field(out, mu=_dev(mu), mode=mode)
        P, G, H = mp.mult_potentials(st.pos, st.q, st.d, st.Q, mu, st.alpha, st.group, st.body, par.eps_in,
                                     par.thole_a, masked=False, same_body_only=same)
        o = out.cpu().numpy().reshape(-1, 10)
        assert _relmax(o[:, 0], P) < 1e-12, mode
        assert _relmax(o[:, 1:4], G) < 1e-12, mode


def test_complex_solvation_fp64(complex_ctx, triple):
    ab, mesh, s = complex_ctx
    ref = triple[1][2]
    r = s.solve(outputs=True)
    assert r["G_diss"] == pytest.approx(ref.G_diss, rel=1e-10)
    assert r["G_vac"] == pytest.approx(ref.G_vac, rel=1e-10)
    assert r["dG_solv_kcal"] == pytest.approx(ref.dG_kcal, rel=1e-10)
    assert np.allclose(r["mu_diss"].reshape(-1, 3), ref.mu_diss, rtol=0, atol=1e-9)


@pytest.mark.parametrize("op", ["fp64_direct", "fp32_tree"])
def test_triple_as_three_systems(bp, triple, op):
    probs, refs = triple
    kw = {} if op == "fp64_direct" else dict(op="fp32_tree", residual_op="fp64_direct", leaf=64, theta=0.5, order=5)
    s = bp.batch_solver(list(probs), **kw)
    assert s.systems() == (3, 4)
    r = s.solve(per_system=True)
    bar = 1e-10 if op == "fp64_direct" else 1e-4
    for q, (ref, sy) in enumerate(zip(refs, r["systems"])):
        assert sy["converged"] == 1
        assert sy["n_panels"] == probs[q].n_panels and sy["n_sites"] == probs[q].sites.n
        assert sy["dG_solv_kcal"] == pytest.approx(ref.dG_kcal, rel=bar), q
    ddg = r["systems"][2]["dG_solv_kcal"] - r["systems"][0]["dG_solv_kcal"] - r["systems"][1]["dG_solv_kcal"]
    ddg_ref = refs[2].dG_kcal - refs[0].dG_kcal - refs[1].dG_kcal
    # each Delta G is within bar of the oracle's, so the difference is within bar * sum |Delta G|
    assert abs(ddg - ddg_ref) <= bar * sum(abs(x.dG_kcal) for x in refs)
    assert r["dG_solv_kcal"] == pytest.approx(sum(x["dG_solv_kcal"] for x in r["systems"]), rel=1e-12)


def test_uneven_batch_matches_separate_solves(bp):
    triples = gen.binding_triples(n_triples=2, subdivs=(3, 4), radius=(6.0, 9.0))
    probs = [p for t in triples for p in t]
    kw = dict(op="fp32_tree", residual_op="fp64_tree", leaf=128, gmres_tol=1e-8, scf_tol=1e-8)
    s = bp.batch_solver(probs, **kw)
    r = s.solve(per_system=True)
    for q, pr in enumerate(probs):
        alone = bp.problem_solver(pr, **kw).solve()
        # same operator, same tolerances: the batch changes only the rounding order
        assert r["systems"][q]["dG_solv_kcal"] == pytest.approx(alone["dG_solv_kcal"], rel=1e-6), q


def test_uneven_batch_matvec_rows_vs_oracle(bp):
    triples = gen.binding_triples(n_triples=2, subdivs=(3, 4), radius=(6.0, 9.0))
    probs = [p for t in triples for p in t]
    s = bp.batch_solver(probs)
    n_tot = sum(p.n_panels for p in probs)
    x = np.random.default_rng(24).normal(size=2 * n_tot)
    y = torch.zeros(2 * n_tot, dtype=torch.float64, device="cuda")
    s.matvec(_dev(x), y, op="fp64_direct")
    yh = y.cpu().numpy()
    off = 0
    rng = np.random.default_rng(25)
    for pr in probs:
        n = pr.n_panels
        par = pr.params
        mesh = bem.build_mesh(pr.verts, pr.tris, par.gauss_k, par.near_factor, body=pr.panel_body)
        xs = np.concatenate([x[off:off + n], x[n_tot + off:n_tot + off + n]])
        rows = np.sort(rng.choice(n, size=6, replace=False))
        y1, y2 = bem.matvec_rows(mesh, xs, rows, par.eps_in, par.eps_out, par.kappa)
        got = np.concatenate([yh[off + rows], yh[n_tot + off + rows]])
        assert _relmax(got, np.concatenate([y1, y2])) < 1e-12
        off += n


def test_body_validation(bp, triple):
    (a, b, ab), _ = triple
    st = ab.sites
    v = np.ascontiguousarray(ab.verts)
    t = np.ascontiguousarray(ab.tris, dtype=np.int32)
    body = np.ascontiguousarray(ab.panel_body, dtype=np.int32)
    s = bp.Solver()
    # missing system id 0
    with pytest.raises(bp.BempolError) as e:
        s.set_mesh(v, t, system=np.ones(ab.n_panels, np.int32))
    assert e.value.status == 1
    # a body that is not closed on its own
    bad = body.copy()
    bad[0] = 1
    with pytest.raises(bp.BempolError) as e:
        s.set_mesh(v, t, body=bad)
    assert e.value.status == 2
    s.set_mesh(v, t, body=body)
    args = [np.ascontiguousarray(x) for x in (st.pos, st.q, st.d, st.Q.reshape(-1, 9), st.alpha)]
    grp = np.ascontiguousarray(st.group, dtype=np.int32)
    sb = np.ascontiguousarray(st.body, dtype=np.int32)
    # plain set_sites is refused on a several-body mesh
    with pytest.raises(bp.BempolError) as e:
        s.set_sites(*args, group=grp)
    assert e.value.status == 8
    # sites out of (system, body) order
    with pytest.raises(bp.BempolError) as e:
        s.set_sites(*args, group=grp, body=np.ascontiguousarray(sb[::-1]))
    assert e.value.status == 3
    # a site of body 0 placed inside body 1
    moved = [x.copy() for x in args]
    moved[0][0] = st.pos[-1] + np.array([0.3, 0.0, 0.0])
    with pytest.raises(bp.BempolError) as e:
        s.set_sites(*moved, group=grp, body=sb)
    assert e.value.status == 3
    s.set_sites(*args, group=grp, body=sb)
