"""Pins for the oracle's Gaussian integrals (McMurchie-Davidson, oracle/md_integrals.c).

Independent references:
* closed forms for s Gaussians: overlap, kinetic, nuclear attraction, (a|b),
  (ab|c), (ab|cd) (Boys F_0 closed form);
* 1D numerical quadrature of overlap factors for any angular momentum;
* higher angular momentum through x_A exp(-a r_A^2) = (1/2a) d/dA_x exp(-a r_A^2),
  evaluated by finite differences of lower-l integrals;
* derivative integrals against finite differences in the atom positions, and
  translational invariance (sum over centres of the derivative vanishes);
* real solid harmonics: orthonormal within a shell, the textbook d forms, and
  rotation invariance of shell-block norms.
"""
import math
import warnings

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import integrals as I
from oracle import basis as OB
from paper_2407_19614_gb300 import workloads as W

rng = np.random.default_rng(1234)


def boys0(T):
    return 1.0 if T < 1e-15 else 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))


def cb_of(shells):
    """shells: list of (l, exponent, centre xyz, atom) -> CBasis with unit coefficients."""
    return I.CBasis([s[0] for s in shells], [s[3] for s in shells], [s[2] for s in shells],
                    [1] * len(shells), [s[1] for s in shells], [1.0] * len(shells))


A = np.array([0.1, -0.3, 0.25])
B = np.array([-0.7, 0.4, 1.1])
C = np.array([0.9, 1.3, -0.6])
Dp = np.array([-0.2, -1.1, 0.5])
a, b, c, d = 0.8, 1.7, 0.45, 2.3


def test_ss_overlap_kinetic_nuclear_closed_form():
    cb = cb_of([(0, a, A, 0), (0, b, B, 1)])
    p, mu = a + b, a * b / (a + b)
    R2 = np.sum((A - B) ** 2)
    S = (math.pi / p) ** 1.5 * math.exp(-mu * R2)
    Tk = mu * (3 - 2 * mu * R2) * S
    P = (a * A + b * B) / p
    Vc = 2 * math.pi / p * math.exp(-mu * R2) * boys0(p * np.sum((P - C) ** 2))
    assert I.one_electron(0, cb)[0, 1] == pytest.approx(S, rel=1e-14)
    assert I.one_electron(1, cb)[0, 1] == pytest.approx(Tk, rel=1e-13)
    V = I.one_electron(2, cb, np.array([3]), C[None, :])
    assert V[0, 1] == pytest.approx(-3 * Vc, rel=1e-13)


def test_two_three_four_centre_s_closed_forms():
    cbx = cb_of([(0, a, A, 0), (0, b, B, 1)])
    R2 = np.sum((A - B) ** 2)
    ref2 = 2 * math.pi ** 2.5 / (a * b * math.sqrt(a + b)) * boys0(a * b / (a + b) * R2)
    assert I.eri2(cbx)[0, 1] == pytest.approx(ref2, rel=1e-14)
    # (ab|c)
    cbp = cb_of([(0, a, A, 0), (0, b, B, 1)])
    cba = cb_of([(0, c, C, 2)])
    p, mu = a + b, a * b / (a + b)
    P = (a * A + b * B) / p
    ref3 = 2 * math.pi ** 2.5 / (p * c * math.sqrt(p + c)) * math.exp(-mu * R2) * boys0(p * c / (p + c) * np.sum((P - C) ** 2))
    t3 = I.eri3(cbp, cba)
    assert t3[0, 1, 0] == pytest.approx(ref3, rel=1e-14)
    assert t3[1, 0, 0] == pytest.approx(ref3, rel=1e-14)
    # (ab|cd)
    cb4 = cb_of([(0, a, A, 0), (0, b, B, 1), (0, c, C, 2), (0, d, Dp, 3)])
    q, nu = c + d, c * d / (c + d)
    Q = (c * C + d * Dp) / q
    ref4 = (2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * math.exp(-mu * R2)
            * math.exp(-nu * np.sum((C - Dp) ** 2)) * boys0(p * q / (p + q) * np.sum((P - Q) ** 2)))
    e4 = I.eri4(cb4)
    assert e4[0, 1, 2, 3] == pytest.approx(ref4, rel=1e-14)
    # 8-fold permutational symmetry
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        assert e4[perm] == pytest.approx(ref4, rel=1e-14)


def _overlap_1d(i, j, x_a, x_b, al, be):
    f = lambda x: (x - x_a) ** i * (x - x_b) ** j * math.exp(-al * (x - x_a) ** 2 - be * (x - x_b) ** 2)
    v, _ = quad(f, -30, 30, epsabs=1e-15, epsrel=1e-13, limit=400)
    return v


@pytest.mark.parametrize("la,lb", [(1, 0), (2, 1), (3, 2), (4, 3)])
def test_overlap_any_l_by_quadrature(la, lb):
    cb = cb_of([(la, a, A, 0), (lb, b, B, 1)])
    S = I.one_electron(0, cb)
    na = (la + 1) * (la + 2) // 2
    for ia, ca in enumerate(OB.cart_components(la)):
        for ib, cbb in enumerate(OB.cart_components(lb)):
            ref = np.prod([_overlap_1d(ca[k], cbb[k], A[k], B[k], a, b) for k in range(3)])
            assert S[ia, na + ib] == pytest.approx(ref, rel=1e-10, abs=1e-14)


def _kinetic_1d_parts(i, j, x_a, x_b, al, be):
    # <i| -1/2 d2/dx2 |j> by quadrature of the analytic second derivative of the j factor
    def g(x):
        u = x - x_b
        e = math.exp(-be * u * u)
        d2 = (j * (j - 1) * u ** (j - 2) if j >= 2 else 0.0) - 2 * be * (2 * j + 1) * u ** j + 4 * be * be * u ** (j + 2)
        return (x - x_a) ** i * math.exp(-al * (x - x_a) ** 2) * d2 * e
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        v, _ = quad(g, -30, 30, epsabs=1e-15, epsrel=1e-13, limit=400)
    return v


@pytest.mark.parametrize("la,lb", [(0, 0), (1, 2), (2, 2), (3, 1)])
def test_kinetic_any_l_by_quadrature(la, lb):
    cb = cb_of([(la, a, A, 0), (lb, b, B, 1)])
    T = I.one_electron(1, cb)
    na = (la + 1) * (la + 2) // 2
    for ia, ca in enumerate(OB.cart_components(la)):
        for ib, cbb in enumerate(OB.cart_components(lb)):
            s = [_overlap_1d(ca[k], cbb[k], A[k], B[k], a, b) for k in range(3)]
            kk = [_kinetic_1d_parts(ca[k], cbb[k], A[k], B[k], a, b) for k in range(3)]
            ref = -0.5 * (kk[0] * s[1] * s[2] + s[0] * kk[1] * s[2] + s[0] * s[1] * kk[2])
            assert T[ia, na + ib] == pytest.approx(ref, rel=1e-9, abs=1e-13)


def _fd5(f, x0, k, h=1e-3):
    def at(s):
        x = x0.copy()
        x[k] += s
        return f(x)
    return (-at(2 * h) + 8 * at(h) - 8 * at(-h) + at(-2 * h)) / (12 * h)


def test_p_functions_from_centre_derivative_of_s_closed_form():
    """(p_x b|c) = 1/(2a) d/dA_x (s b|c), with the s integral in closed form."""
    p_ = a + b

    def ss_c(Avec):
        mu = a * b / p_
        P = (a * Avec + b * B) / p_
        return (2 * math.pi ** 2.5 / (p_ * c * math.sqrt(p_ + c)) * math.exp(-mu * np.sum((Avec - B) ** 2))
                * boys0(p_ * c / (p_ + c) * np.sum((P - C) ** 2)))

    t3 = I.eri3(cb_of([(1, a, A, 0), (0, b, B, 1)]), cb_of([(0, c, C, 2)]))
    for k in range(3):
        ref = _fd5(ss_c, A.copy(), k) / (2 * a)
        assert t3[k, 3, 0] == pytest.approx(ref, rel=1e-9)

    def s_s2(Cvec):
        return 2 * math.pi ** 2.5 / (a * c * math.sqrt(a + c)) * boys0(a * c / (a + c) * np.sum((A - Cvec) ** 2))

    m2 = I.eri2(cb_of([(0, a, A, 0), (1, c, C, 1)]))
    for k in range(3):
        assert m2[0, 1 + k] == pytest.approx(_fd5(s_s2, C.copy(), k) / (2 * c), rel=1e-9)


def test_d_functions_from_centre_derivative_of_p():
    """x_A^2 e = (d/dA_x [x_A e] + e)/(2a);  x_A y_A e = d/dA_y [x_A e]/(2a)."""
    aux = cb_of([(2, c, C, 2)])

    def p_block(Avec):
        return I.eri3(cb_of([(1, a, Avec, 0), (1, b, B, 1)]), aux)

    d_blk = I.eri3(cb_of([(2, a, A, 0), (1, b, B, 1)]), aux)    # rows: d(6) then p(3)
    s_blk = I.eri3(cb_of([(0, a, A, 0), (1, b, B, 1)]), aux)
    h = 1e-3

    def dA(k):
        out = []
        for s in (2 * h, h, -h, -2 * h):
            Av = A.copy()
            Av[k] += s
            out.append(p_block(Av))
        return (-out[0] + 8 * out[1] - 8 * out[2] + out[3]) / (12 * h)

    dx = dA(0)
    dy = dA(1)
    # d order: xx, xy, xz, yy, yz, zz; p rows 0..2 = x,y,z; partner p at rows 3..5 (d) / 6..8
    xx = (dx[0, 3:6, :] + s_blk[0, 1:4, :]) / (2 * a)
    xy = dy[0, 3:6, :] / (2 * a)
    assert np.allclose(d_blk[0, 6:9, :], xx, rtol=1e-8, atol=1e-12)
    assert np.allclose(d_blk[1, 6:9, :], xy, rtol=1e-8, atol=1e-12)


def test_derivative_integrals_match_finite_differences():
    mol = W.water_monomer(3)
    basis = OB.AOBasis(mol.primary[:6] + mol.primary[6:9], mol.xyz)
    auxb = OB.AOBasis([s for s in mol.aux if s.l <= 3][:14] + [s for s in mol.aux if s.atom == 1][:5], mol.xyz)

    def ints(xyz):
        b2 = OB.AOBasis(basis.shells, xyz)
        x2 = OB.AOBasis(auxb.shells, xyz)
        return (I.one_electron(0, b2.cb), I.one_electron(1, b2.cb),
                I.one_electron(2, b2.cb, mol.Z, xyz), I.eri2(x2.cb), I.eri3(b2.cb, x2.cb))

    h = 1e-4
    for atom, dim in [(0, 2), (1, 0), (2, 1)]:
        xp, xm = mol.xyz.copy(), mol.xyz.copy()
        xp[atom, dim] += h
        xm[atom, dim] -= h
        Ip, Im = ints(xp), ints(xm)
        an = (I.one_electron(0, basis.cb, datom=atom, ddim=dim), I.one_electron(1, basis.cb, datom=atom, ddim=dim),
              I.one_electron(2, basis.cb, mol.Z, mol.xyz, datom=atom, ddim=dim),
              I.eri2(auxb.cb, datom=atom, ddim=dim), I.eri3(basis.cb, auxb.cb, datom=atom, ddim=dim))
        for k in range(5):
            fd = (Ip[k] - Im[k]) / (2 * h)
            scale = max(1.0, np.abs(an[k]).max())
            assert np.abs(fd - an[k]).max() < 2e-6 * scale, (atom, dim, k, np.abs(fd - an[k]).max())


def test_derivative_translational_invariance():
    mol = W.water_monomer(4)
    basis = OB.AOBasis(mol.primary, mol.xyz)
    auxb = OB.AOBasis(mol.aux, mol.xyz)
    for dim in range(3):
        s3 = sum(I.eri3(basis.cb, auxb.cb, datom=at, ddim=dim) for at in range(3))
        s2 = sum(I.eri2(auxb.cb, datom=at, ddim=dim) for at in range(3))
        sS = sum(I.one_electron(0, basis.cb, datom=at, ddim=dim) for at in range(3))
        sV = sum(I.one_electron(2, basis.cb, mol.Z, mol.xyz, datom=at, ddim=dim) for at in range(3))
        assert np.abs(s3).max() < 1e-11
        assert np.abs(s2).max() < 1e-11
        assert np.abs(sS).max() < 1e-13
        assert np.abs(sV).max() < 1e-11


@pytest.mark.parametrize("l", range(0, 5))
def test_spherical_functions_orthonormal_within_shell(l):
    sh = [W.Shell(0, l, [0.7], [1.0])]
    bas = OB.AOBasis(sh, np.zeros((1, 3)), pure=True)
    S = bas.to_ao2(I.one_electron(0, bas.cb))
    assert S.shape == (2 * l + 1, 2 * l + 1)
    assert np.allclose(S, np.eye(2 * l + 1), atol=1e-13)


def test_d_solid_harmonics_textbook_forms():
    M = OB.solid_harmonic_coeffs(2)        # rows m = -2..2 ; cols xx, xy, xz, yy, yz, zz
    forms = {
        -2: [0, 1, 0, 0, 0, 0],     # xy
        -1: [0, 0, 0, 0, 1, 0],     # yz
        0: [-1, 0, 0, -1, 0, 2],    # 2z^2 - x^2 - y^2
        1: [0, 0, 1, 0, 0, 0],      # xz
        2: [1, 0, 0, -1, 0, 0],     # x^2 - y^2
    }
    for row, m in enumerate(range(-2, 3)):
        f = np.array(forms[m], dtype=float)
        v = M[row]
        k = np.argmax(np.abs(f))
        ratio = v[k] / f[k]
        assert ratio > 0
        assert np.allclose(v, ratio * f, atol=1e-14)


def _rot(axis, ang):
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def test_rotation_invariance_of_spherical_shell_blocks():
    mol = W.water_monomer(1)
    R = _rot(np.array([0.3, -0.5, 0.8]), 1.1)
    out = []
    for xyz in (mol.xyz, mol.xyz @ R.T + np.array([0.4, -1.0, 2.0])):
        bas = OB.AOBasis(mol.primary, xyz, pure=True)
        aux = OB.AOBasis(mol.aux, xyz, pure=True)
        raw = I.eri3(bas.cb, aux.cb)
        t = np.einsum("am,bn,cp,mnp->abc", bas.T, bas.T, aux.T, raw, optimize=True)
        norms = {}
        for i in range(len(mol.primary)):
            for j in range(len(mol.primary)):
                for k in range(len(mol.aux)):
                    blk = t[np.ix_(bas.ao_shell == i, bas.ao_shell == j, aux.ao_shell == k)]
                    norms[(i, j, k)] = np.linalg.norm(blk)
        out.append(norms)
    for key in out[0]:
        assert out[1][key] == pytest.approx(out[0][key], rel=1e-9, abs=1e-14)
