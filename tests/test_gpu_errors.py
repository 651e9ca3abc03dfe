"""Input validation and error reporting through the C ABI (host-side checks; no faults)."""
import numpy as np
import pytest

import gen

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


def _sites(pos):
    n = pos.shape[0]
    return (np.ascontiguousarray(pos), np.zeros(n), np.zeros((n, 3)), np.zeros((n, 9)), np.zeros(n))


def test_state_order(bp):
    s = bp.Solver()
    with pytest.raises(bp.BempolError) as e:
        s.solve()
    assert e.value.status == 8
    with pytest.raises(bp.BempolError) as e:
        s.set_sites(*_sites(np.zeros((1, 3))))
    assert e.value.status == 8


def test_open_and_bad_meshes(bp):
    v, f = gen.icosphere(4.0, 1)
    s = bp.Solver()
    with pytest.raises(bp.BempolError) as e:
        s.set_mesh(v, np.ascontiguousarray(f[:-1]))        # a hole
    assert e.value.status == 2
    g = f.copy()
    g[0] = g[0][[0, 2, 1]]                                  # one panel flipped
    with pytest.raises(bp.BempolError) as e:
        s.set_mesh(v, g)
    assert e.value.status == 2
    g = f.copy()
    g[3, 1] = v.shape[0] + 5                                # index out of range
    with pytest.raises(bp.BempolError) as e:
        s.set_mesh(v, g)
    assert e.value.status == 2


def test_bad_sites(bp):
    v, f = gen.icosphere(4.0, 2)
    s = bp.Solver()
    s.set_mesh(v, f)
    with pytest.raises(bp.BempolError) as e:                # outside
        s.set_sites(*_sites(np.array([[0.0, 0.0, 0.0], [5.0, 0.0, 0.0]])))
    assert e.value.status == 3
    with pytest.raises(bp.BempolError) as e:                # on the surface
        s.set_sites(*_sites(np.array([[0.0, 0.0, 3.98]])))
    assert e.value.status == 3
    pos, q, d, Q, a = _sites(np.array([[0.5, 0.0, 0.0]]))
    Q[0, 0] = 1.0                                           # not traceless
    with pytest.raises(bp.BempolError) as e:
        s.set_sites(pos, q, d, Q, a)
    assert e.value.status == 3
    a[0] = -1.0
    Q[:] = 0
    with pytest.raises(bp.BempolError) as e:                # negative polarizability
        s.set_sites(pos, q, d, Q, a)
    assert e.value.status == 3
    a[0] = 1.0
    s.set_sites(pos, q, d, Q, a)                            # and a valid one passes


def test_not_converged_is_reported(bp):
    pr = gen.with_params(gen.sphere_r4_1280(), scf_maxit=2)
    s = bp.problem_solver(pr)
    out = s.solve(allow_unconverged=True)
    assert out["status"] == 4
    assert out["scf_iters_diss"] == 2
    with pytest.raises(bp.BempolError):
        s.solve()
