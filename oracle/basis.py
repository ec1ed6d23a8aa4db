"""Basis-set bookkeeping for the oracle -- TEST INFRASTRUCTURE ONLY.

* Primitive normalisation of x^l exp(-a r^2):
      N(a, l) = [ (4a)^l (2a/pi)^{3/2} / (2l-1)!! ]^{1/2},
  then each contracted function is renormalised numerically from its own
  overlap (so contracted shells are normalised whatever the coefficients).
* Real solid harmonics S_lm, m = -l..l, from the closed-form expansion in
  Cartesian monomials (Helgaker, Joergensen, Olsen, Eqs. 6.4.47-6.4.50):
      S_lm = sum_{t,u,v} C^{lm}_{tuv} x^{2t+|m|-2(u+v)} y^{2(u+v)} z^{l-2t-|m|},
      C^{lm}_{tuv} = (-1)^{t+v-v_m} (1/4)^t C(l,t) C(l-t,|m|+t) C(t,u) C(|m|,2v),
  v_m = 0 (m >= 0) or 1/2 (m < 0); every spherical function is then scaled to
  unit self-overlap.  Spherical ordering within a shell is m = -l..l; Cartesian
  ordering is lx = l..0, ly = l-lx..0.
"""

from __future__ import annotations

from math import comb, pi, sqrt

import numpy as np

from . import integrals as I


def cart_components(l):
    return [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]


def dfact(n):
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


def prim_norm(a, l):
    return sqrt((4 * a) ** l * (2 * a / pi) ** 1.5 / dfact(2 * l - 1))


def solid_harmonic_coeffs(l):
    """(2l+1, ncart(l)) unnormalised coefficients of S_lm in Cartesian monomials."""
    comps = cart_components(l)
    index = {c: k for k, c in enumerate(comps)}
    M = np.zeros((2 * l + 1, len(comps)))
    for row, m in enumerate(range(-l, l + 1)):
        am = abs(m)
        two_vm = 0 if m >= 0 else 1
        # v runs over v_m, v_m+1, ..., floor(|m|/2 - v_m) + v_m ; track 2v
        vmax2 = 2 * int((am - two_vm) // 2) + two_vm
        for t in range((l - am) // 2 + 1):
            for u in range(t + 1):
                for v2 in range(two_vm, vmax2 + 1, 2):
                    sign_exp = t + (v2 - two_vm) // 2
                    c = (-1) ** sign_exp * 0.25 ** t * comb(l, t) * comb(l - t, am + t) * comb(t, u) * comb(am, v2)
                    ex = 2 * t + am - 2 * u - v2
                    ey = 2 * u + v2
                    ez = l - 2 * t - am
                    M[row, index[(ex, ey, ez)]] += c
    return M


class AOBasis:
    """A list of shells on atoms -> Cartesian C-basis plus AO transform matrix."""

    def __init__(self, shells, atom_xyz, pure=True):
        self.shells = shells
        self.pure = pure
        xyz = np.array([atom_xyz[s.atom] for s in shells]).reshape(-1, 3)
        exps, coefs, nprim = [], [], []
        for s in shells:
            nprim.append(len(s.exps))
            for a, d in zip(s.exps, s.coefs):
                exps.append(a)
                coefs.append(d * prim_norm(a, s.l))
        self.cb = I.CBasis([s.l for s in shells], [s.atom for s in shells], xyz, nprim, exps, coefs)
        S = I.one_electron(0, self.cb)
        blocks, ao_atom, ao_shell, off = [], [], [], 0
        self.shell_off = []
        for k, s in enumerate(shells):
            nc = (s.l + 1) * (s.l + 2) // 2
            Sc = S[off:off + nc, off:off + nc]
            if pure:
                M = solid_harmonic_coeffs(s.l)
            else:
                M = np.eye(nc)
            norms = np.sqrt(np.einsum("ma,ab,mb->m", M, Sc, M))
            M = M / norms[:, None]
            blocks.append(M)
            self.shell_off.append(sum(b.shape[0] for b in blocks[:-1]))
            ao_atom += [s.atom] * M.shape[0]
            ao_shell += [k] * M.shape[0]
            off += nc
        nao = sum(b.shape[0] for b in blocks)
        self.T = np.zeros((nao, self.cb.ncart))
        r = c = 0
        for M in blocks:
            self.T[r:r + M.shape[0], c:c + M.shape[1]] = M
            r += M.shape[0]
            c += M.shape[1]
        self.nao = nao
        self.ao_atom = np.array(ao_atom)
        self.ao_shell = np.array(ao_shell)

    def to_ao2(self, M):
        return self.T @ M @ self.T.T
