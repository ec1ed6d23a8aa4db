"""RI-HF energy and analytic gradient, plain numpy FP64 -- TEST INFRASTRUCTURE ONLY.

Follows the paper (Stocks, Palethorpe, Barca) section by section:

* Sec. 2.2, Eq. ri_eri:   (mu nu|lam sig) ~ sum_PQ (mu nu|P) A^{-1}_PQ (lam sig|Q)
* Eqs. symmetric_ri/biap: A = (P|Q) = L L^T (Cholesky, lower L); the paper's
                          A^L is read as L^{-T}, so B^P_{mu nu} = (L^{-1} T)_P with
                          T_P = (mu nu|P) and A^{-1} = L^{-T} L^{-1}.
* Eq. fock_split:         F = h + J + K
* Eq. j_ri:               J_{mu nu} = sum_P B^P_{mu nu} sum_{lam sig} B^P_{lam sig} D_{lam sig}
* Eqs. k_ri_2, tp:        K_{mu nu} = -sum_{iP} B^P_{i mu} B^P_{i nu},
                          B^P_{i mu} = sum_sig B^P_{mu sig} C_{sig i}
* Roothaan FC = SC eps,   D = 2 sum_i C_{mu i} C_{nu i},  E = 1/2 Tr D(h+F) + V_nn
* Eq. rihf_gradient:      E^xi = sum D h^xi - sum W S^xi + sum Y^P (mu nu|P)^xi
                                 - 1/2 sum Z_PQ (P|Q)^xi  (+ V_nn^xi)
  with, for C~ = sqrt(2) C_occ (so D = C~ C~^T),
      c_P  = sum_Q A^{-1}_PQ sum D (mu nu|Q)              (the paper's L^P)
      X^P_ij = sum_Q A^{-1}_PQ (C~^T T_Q C~)_ij
      Y^P  = D c_P - 1/2 C~ X^P C~^T
      Z_PQ = c_P c_Q - 1/2 sum_ij X^P_ij X^Q_ij
      W    = 2 sum_i eps_i C_{mu i} C_{nu i}
  The scaling C -> C~ is the reading under which the printed 1/2 factors and
  L^P = sum_i X^P_ii hold together; finite differences pin it (tests).

SCF control (the paper states only "standard", Sec. 3.1): canonical
orthogonalisation X = U s^{-1/2} over overlap eigenvalues s > 1e-8, core-
Hamiltonian or caller-supplied orbital guess, Pulay commutator DIIS in the
orthonormal basis (e = X^T (F D S - S D F) X, up to 8 vectors), aufbau
occupation, convergence when max|e| < conv_diis and |dE| < conv_e.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import integrals as I
from .basis import AOBasis


class System:
    """All geometry-dependent integrals of one molecule in the AO basis."""

    def __init__(self, mol, pure=True, need_eri3=True):
        self.mol = mol
        self.Z = np.asarray(mol.Z, dtype=np.int32)
        self.xyz = np.asarray(mol.xyz, dtype=np.float64)
        self.pure = pure
        self.bas = AOBasis(mol.primary, self.xyz, pure)
        self.aux = AOBasis(mol.aux, self.xyz, pure) if mol.aux else None
        self.nao = self.bas.nao
        self.nocc = int(self.Z.sum()) // 2
        tb = self.bas
        self.S = tb.to_ao2(I.one_electron(0, tb.cb))
        self.Tkin = tb.to_ao2(I.one_electron(1, tb.cb))
        self.V = tb.to_ao2(I.one_electron(2, tb.cb, self.Z, self.xyz))
        self.h = self.Tkin + self.V
        self.Vnn = nuclear_repulsion(self.Z, self.xyz)
        if self.aux is not None:
            self.A = self.aux.to_ao2(I.eri2(self.aux.cb))
            self.naux = self.aux.nao
            if need_eri3:
                self.T3 = self.eri3_ao()

    def eri3_ao(self, datom=-1, ddim=0):
        """(mu nu|P) in the AO bases, returned as T[P, mu, nu]."""
        raw = I.eri3(self.bas.cb, self.aux.cb, datom, ddim)
        t = np.tensordot(raw, self.aux.T, axes=([2], [1]))          # (a, b, P)
        t = np.tensordot(self.bas.T, t, axes=([1], [0]))             # (mu, b, P)
        t = np.tensordot(t, self.bas.T, axes=([1], [1]))             # (mu, P, nu)
        return np.ascontiguousarray(t.transpose(1, 0, 2))


def nuclear_repulsion(Z, xyz):
    e = 0.0
    for a in range(len(Z)):
        for b in range(a):
            e += Z[a] * Z[b] / np.linalg.norm(xyz[a] - xyz[b])
    return e


def nuclear_repulsion_grad(Z, xyz):
    g = np.zeros_like(xyz)
    for a in range(len(Z)):
        for b in range(len(Z)):
            if a != b:
                r = xyz[a] - xyz[b]
                g[a] -= Z[a] * Z[b] * r / np.linalg.norm(r) ** 3
    return g


def cholesky_fit(A, T3):
    """A = L L^T; B = L^{-1} T (forward substitution over the auxiliary index)."""
    L = np.linalg.cholesky(A)
    naux = A.shape[0]
    B = sla.solve_triangular(L, T3.reshape(naux, -1), lower=True).reshape(T3.shape)
    return L, B


def density(C_occ):
    return 2.0 * C_occ @ C_occ.T


def coulomb_ri(B, D):
    naux, n, _ = B.shape
    Bf = B.reshape(naux, n * n)
    d = Bf @ D.reshape(-1)                           # d_P = sum_{lam sig} B^P D
    return (d @ Bf).reshape(n, n)                    # J = sum_P d_P B^P


def exchange_ri(B, C_occ):
    naux, n, _ = B.shape
    H = (B.reshape(naux * n, n) @ C_occ).reshape(naux, n, -1)    # B^P_{mu i}, Eq. tp
    Hm = H.transpose(1, 0, 2).reshape(n, -1)                      # rows mu, columns (P, i)
    return -(Hm @ Hm.T)                                           # Eq. k_ri_2


def exchange_density_ri(B, D):
    """Eq. k_ri_1: K = -1/2 sum_{lam sig} D_{lam sig} sum_P B^P_{mu sig} B^P_{lam nu}."""
    return -0.5 * np.einsum("ls,pms,pln->mn", D, B, B)


def canonical_orthogonaliser(S, thresh=1e-8):
    s, U = np.linalg.eigh(S)
    keep = s > thresh
    return U[:, keep] / np.sqrt(s[keep])


class SCFResult:
    pass


def spherical_average(F, labels):
    """Rotation average of a matrix over real solid harmonics: labels[i] =
    (first function of i's shell, l, m index).  Entries between different l or
    m vanish; for equal l and m the mean over m of the shell pair's (m, m)
    entries remains."""
    n = F.shape[0]
    out = np.zeros_like(F)
    for i in range(n):
        a, li, mi = labels[i]
        for j in range(n):
            b, lj, mj = labels[j]
            if li == lj and mi == mj:
                out[i, j] = np.mean([F[a + m, b + m] for m in range(2 * li + 1)])
    return out


def sph_labels(shells):
    """(first function of the shell, l, m index) per spherical function."""
    out, k = [], 0
    for sh in shells:
        for m in range(2 * sh.l + 1):
            out.append((k, sh.l, m))
        k += 2 * sh.l + 1
    return out


def occupied_by_l(C, eps, labels, occ_l):
    """Columns of C reordered so that the occupied ones follow occ_l (the l of
    each occupied orbital, in order): for every l, the lowest-eps columns whose
    weight lies in functions of that l.  The spherical average makes every
    eigenvector pure in l; a configuration such as 1s2 2s2 2p4 then fixes which
    orbitals carry which occupation even where the basis puts 2p below 2s."""
    lcol = [labels[int(np.argmax(np.abs(C[:, j])))][1] for j in range(C.shape[1])]
    order = list(np.argsort(eps, kind="stable"))
    chosen = []
    for l in occ_l:
        j = next(j for j in order if lcol[j] == l and j not in chosen)
        chosen.append(j)
    rest = [j for j in order if j not in chosen]
    idx = chosen + rest
    return C[:, idx], eps[idx]


def scf(h, S, Vnn, nocc, fock_2e, C_guess=None, max_iter=128, conv_e=1e-11, conv_diis=1e-10, diis_size=8,
        occ=None, sph=None, occ_l=None):
    """Closed-shell Roothaan SCF.  fock_2e(C_occ, D) -> J + K.

    occ: occupation numbers n_i of the len(occ) lowest orbitals (the
    spherically averaged atoms of the SAD guess); the closed-shell formulas
    then hold with C_occ -> C_occ diag(sqrt(n_i / 2)), i.e. D = sum_i n_i C_i C_i^T
    and K = -1/2 sum_P sum_i n_i (B^P C_i)(B^P C_i)^T.  None: n_i = 2.
    sph: labels of sph_labels; every Fock matrix is then replaced by its
    spherical average (an isolated atom with a spherically symmetric density).
    occ_l (with sph): the l of each occupied orbital; occupation then follows
    the configuration instead of the eigenvalue order (occupied_by_l)."""
    w = None
    if occ is not None:
        nocc = len(occ)
        w = np.sqrt(np.asarray(occ, dtype=np.float64) / 2.0)
    X = canonical_orthogonaliser(S)
    def orbitals(Fm):
        e, Cp = np.linalg.eigh(X.T @ Fm @ X)
        C = X @ Cp
        if occ_l is not None:
            C, e = occupied_by_l(C, e, sph, occ_l)
        return e, C

    if C_guess is None:
        e, C = orbitals(h)
    else:
        C = np.array(C_guess, dtype=np.float64)
    Fs, Es = [], []
    E_old = None
    res = SCFResult()
    res.converged = False
    for it in range(1, max_iter + 1):
        Co = C[:, :nocc] if w is None else C[:, :nocc] * w
        D = density(Co)
        F = h + fock_2e(Co, D)
        if sph is not None:
            F = spherical_average(F, sph)
        E = 0.5 * np.sum(D * (h + F)) + Vnn
        err = X.T @ (F @ D @ S - S @ D @ F) @ X
        Fs.append(F)
        Es.append(err)
        if len(Fs) > diis_size:
            Fs.pop(0)
            Es.pop(0)
        emax = np.abs(err).max()
        if E_old is not None and abs(E - E_old) < conv_e and emax < conv_diis:
            res.converged = True
            res.iterations = it
            break
        E_old = E
        m = len(Fs)
        if m >= 2:
            Bm = -np.ones((m + 1, m + 1))
            Bm[m, m] = 0.0
            for i in range(m):
                for j in range(m):
                    Bm[i, j] = np.sum(Es[i] * Es[j])
            rhs = np.zeros(m + 1)
            rhs[m] = -1.0
            coef = np.linalg.solve(Bm, rhs)[:m]
            Fx = sum(c * f for c, f in zip(coef, Fs))
        else:
            Fx = F
        eps, C = orbitals(Fx)
    else:
        res.iterations = max_iter
    # Final orbitals diagonalise the converged (unextrapolated) Fock matrix.
    eps, res.C = orbitals(F)
    res.eps = eps
    res.D = density(res.C[:, :nocc] if w is None else res.C[:, :nocc] * w)
    res.F = F
    res.E = E
    res.max_err = emax
    return res


def rihf_energy(sysm, C_guess=None, **kw):
    L, B = cholesky_fit(sysm.A, sysm.T3)

    def f2(Co, D):
        return coulomb_ri(B, D) + exchange_ri(B, Co)

    r = scf(sysm.h, sysm.S, sysm.Vnn, sysm.nocc, f2, C_guess=C_guess, **kw)
    r.L, r.B = L, B
    return r


def hf4c_energy(sysm, C_guess=None, **kw):
    """Brute-force four-centre HF (Eqs. fock_build, j, k) for tiny bases."""
    raw = I.eri4(sysm.bas.cb)
    T = sysm.bas.T
    eri = np.einsum("ai,bj,ck,dl,ijkl->abcd", T, T, T, T, raw, optimize=True)

    def f2(Co, D):
        J = np.einsum("mnls,ls->mn", eri, D)
        K = -0.5 * np.einsum("msln,ls->mn", eri, D)
        return J + K

    r = scf(sysm.h, sysm.S, sysm.Vnn, sysm.nocc, f2, C_guess=C_guess, **kw)
    r.eri = eri
    return r


def rihf_gradient_terms(sysm, res, atoms=None):
    """dE/dR (natoms, 3) by Eq. rihf_gradient, and its pieces.  With `atoms`
    (a list of atom indices) only those atoms' rows are evaluated; the others
    stay zero."""
    nocc = sysm.nocc
    Ct = np.sqrt(2.0) * res.C[:, :nocc]
    D = Ct @ Ct.T
    W = Ct @ np.diag(res.eps[:nocc]) @ Ct.T
    A = sysm.A
    T3 = sysm.T3
    cho = sla.cho_factor(A, lower=True)
    dtil = np.einsum("pmn,mn->p", T3, D)
    c = sla.cho_solve(cho, dtil)                                  # L^P of the paper
    Tij = np.einsum("mi,pmn,nj->pij", Ct, T3, Ct)                  # (ij|P) with C~
    X = sla.cho_solve(cho, Tij.reshape(sysm.naux, -1)).reshape(Tij.shape)
    Y = D[None, :, :] * c[:, None, None] - 0.5 * np.einsum("mi,pij,nj->pmn", Ct, X, Ct)
    Z = np.outer(c, c) - 0.5 * np.einsum("pij,qij->pq", X, X)
    natoms = len(sysm.Z)
    g1, gS, g3, g2 = (np.zeros((natoms, 3)) for _ in range(4))
    tb, ta = sysm.bas, sysm.aux
    for a in range(natoms) if atoms is None else atoms:
        for d in range(3):
            dT = tb.to_ao2(I.one_electron(1, tb.cb, datom=a, ddim=d))
            dV = tb.to_ao2(I.one_electron(2, tb.cb, sysm.Z, sysm.xyz, datom=a, ddim=d))
            dS = tb.to_ao2(I.one_electron(0, tb.cb, datom=a, ddim=d))
            dA = ta.to_ao2(I.eri2(ta.cb, datom=a, ddim=d))
            dT3 = sysm.eri3_ao(datom=a, ddim=d)
            g1[a, d] = np.sum(D * (dT + dV))
            gS[a, d] = -np.sum(W * dS)
            g3[a, d] = np.sum(Y * dT3)
            g2[a, d] = -0.5 * np.sum(Z * dA)
    gnn = nuclear_repulsion_grad(sysm.Z, sysm.xyz)
    out = SCFResult()
    out.grad = g1 + gS + g3 + g2 + gnn
    out.parts = dict(one=g1, overlap=gS, three=g3, two=g2, nuc=gnn)
    out.Y, out.Z, out.c, out.X, out.W = Y, Z, c, X, W
    return out


def energy_at(mol, xyz, pure=True, **kw):
    """RI-HF energy of ``mol`` moved to coordinates ``xyz`` (bohr)."""
    import copy

    m2 = copy.copy(mol)
    m2.xyz = np.array(xyz, dtype=np.float64)
    return rihf_energy(System(m2, pure=pure), **kw).E
