"""dfjk_coulomb_gradient and dfjk_jk_gradient against the oracle's
finite-difference gradients of E_J = u^T V^-1 u / 2 and E_K (density held
fixed): FP64 and mixed handles, a density that is not C C^T, one atom (zero
gradient), one occupied orbital (E_J = E_K), translation invariance."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2404_09452_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2404_09452_gb300 import dfjk  # noqa: E402

# Richardson-extrapolated central differences are good to ~1e-9 here; the
# analytic gradient is FP64 throughout.
GRAD_TOL = 1e-7


def _density(m, seed=3000):
    S = O.overlap(m.orb, m.coords)
    C = I.orthonormalize(I.c_occ_raw(m.nao, I.default_nocc(m.nao), seed), S)
    return C @ C.T


def _check(m, D, precision):
    h = dfjk.Handle(m, precision=precision)
    g = h.coulomb_gradient(torch.from_numpy(D).cuda()).cpu().numpy()
    h.close()
    ref = O.coulomb_gradient_fd(m.orb, m.aux, m.coords, D)
    err = np.max(np.abs(g - ref))
    assert err < GRAD_TOL * max(1.0, np.abs(ref).max()), (err, g, ref)
    assert np.max(np.abs(g.sum(axis=0))) < 1e-10 * max(1.0, np.abs(g).max())
    return g


@pytest.mark.parametrize("precision", [dfjk.DFJK_FP64, dfjk.DFJK_MIXED])
def test_gradient_water(precision):
    m = I.water()
    _check(m, _density(m), precision)


@pytest.mark.parametrize("precision", [dfjk.DFJK_FP64, dfjk.DFJK_MIXED])
def test_gradient_six_atoms(precision):
    m = I.molecule(6, seed=1006)
    _check(m, _density(m), precision)


def test_gradient_indefinite_density():
    m = I.molecule(4, seed=1004)
    S = O.overlap(m.orb, m.coords)
    C = I.orthonormalize(I.c_occ_raw(m.nao, I.default_nocc(m.nao), 3001), S)
    n = C.shape[1]
    D = C[:, : n // 2] @ C[:, : n // 2].T - 0.5 * C[:, n // 2 :] @ C[:, n // 2 :].T
    _check(m, D, dfjk.DFJK_FP64)


def test_gradient_single_atom_is_zero():
    m = I.molecule(1, seed=1001)
    h = dfjk.Handle(m, precision=dfjk.DFJK_FP64)
    g = h.coulomb_gradient(torch.from_numpy(_density(m)).cuda()).cpu().numpy()
    h.close()
    assert g.shape == (1, 3) and np.max(np.abs(g)) < 1e-10


def _orbitals(m, nocc=None, seed=3000):
    S = O.overlap(m.orb, m.coords)
    return I.orthonormalize(I.c_occ_raw(m.nao, nocc or I.default_nocc(m.nao), seed), S)


@pytest.mark.parametrize("precision", [dfjk.DFJK_FP64, dfjk.DFJK_MIXED])
@pytest.mark.parametrize("natom", [3, 6])
def test_jk_gradient(precision, natom):
    m = I.water() if natom == 3 else I.molecule(natom, seed=1000 + natom)
    C = _orbitals(m)
    D = C @ C.T
    h = dfjk.Handle(m, precision=precision)
    Cd = torch.from_numpy(C).cuda()
    gk = h.jk_gradient(Cd, 0.0, 1.0).cpu().numpy()
    gjk = h.jk_gradient(Cd, 1.0, -0.5).cpu().numpy()
    gj = h.jk_gradient(Cd, 1.0, 0.0).cpu().numpy()
    gj_density = h.coulomb_gradient(torch.from_numpy(D).cuda()).cpu().numpy()
    h.close()
    refk = O.exchange_gradient_fd(m.orb, m.aux, m.coords, D)
    refj = O.coulomb_gradient_fd(m.orb, m.aux, m.coords, D)
    scale = max(1.0, np.abs(refk).max())
    assert np.max(np.abs(gk - refk)) < GRAD_TOL * scale, (gk, refk)
    assert np.max(np.abs(gjk - (refj - 0.5 * refk))) < GRAD_TOL * scale
    assert np.max(np.abs(gj - gj_density)) < 1e-12 * max(1.0, np.abs(gj).max())
    assert np.max(np.abs(gk.sum(axis=0))) < 1e-10 * scale


def test_jk_gradient_one_orbital_cancels():
    """One occupied orbital: E_K = E_J at every geometry, so the gradient of
    E_J - E_K vanishes."""
    m = I.molecule(4, seed=1004)
    C = _orbitals(m, nocc=1, seed=3002)
    h = dfjk.Handle(m, precision=dfjk.DFJK_FP64)
    Cd = torch.from_numpy(C).cuda()
    g = h.jk_gradient(Cd, 1.0, -1.0).cpu().numpy()
    gj = h.jk_gradient(Cd, 1.0, 0.0).cpu().numpy()
    h.close()
    assert np.abs(gj).max() > 1e-3
    assert np.max(np.abs(g)) < 1e-11 * np.abs(gj).max()


def test_jk_gradient_sampled_20_atoms():
    """20 atoms (nao 300, naux 720), the mixed handle: three components of the
    gradient of E_J - E_K/2 against central differences of the oracle's
    energies, one component at a time; the rest by the translation sum rule."""
    m = I.molecule(20, seed=1020)
    C = _orbitals(m)
    D = C @ C.T
    h = dfjk.Handle(m, precision=dfjk.DFJK_MIXED)
    g = h.jk_gradient(torch.from_numpy(C).cuda(), 1.0, -0.5).cpu().numpy()
    h.close()
    assert np.max(np.abs(g.sum(axis=0))) < 1e-10 * np.abs(g).max()
    for a, x in ((0, 0), (7, 1), (13, 2)):
        d = []
        for step in (2e-3, 1e-3):
            e = []
            for sgn in (1, -1):
                c = m.coords.copy()
                c[a, x] += sgn * step
                ej, ek = O.energies_geometry(m.orb, m.aux, c, D)
                e.append(ej - 0.5 * ek)
            d.append((e[0] - e[1]) / (2 * step))
        ref = (4 * d[1] - d[0]) / 3
        assert abs(g[a, x] - ref) < GRAD_TOL * max(1.0, abs(ref)), (a, x, g[a, x], ref)


def test_coulomb_gradient_fp32_pairs():
    """The mixed handle's Coulomb gradient evaluates the pairs below the FP32
    threshold in FP32 (as its build does their integrals): against the FP64
    handle at 20 atoms the difference stays at the level of the integrals'."""
    m = I.molecule(20, seed=1020)
    D = torch.from_numpy(_density(m)).cuda()
    h64 = dfjk.Handle(m, precision=dfjk.DFJK_FP64)
    g64 = h64.coulomb_gradient(D).cpu().numpy()
    h64.close()
    hm = dfjk.Handle(m, precision=dfjk.DFJK_MIXED)
    assert hm.npair_fp32 > 0
    gm = hm.coulomb_gradient(D).cpu().numpy()
    hm.close()
    err = np.max(np.abs(gm - g64))
    assert err < 1e-8 * max(1.0, np.abs(g64).max()), err
