"""Oracle (test infrastructure only) for the learned SCF guess: a plain FP64
numpy statement of the elementwise two-layer network, its loss gradient, one
Adam step, BF16 rounding and the per-element features.

Only tests, __graft_entry__.smoke() and bench.py's CPU baseline use this module.

The network (the learned-guess design of the method's AIMD driver; the paper's
own guess reuses the previous orbitals, Sec. 3.3): for features x (12),
    z = W1 x + b1,   h = tanh(z),   y = w2 . h + b2,
loss L = (1/M) sum_e (y_e - t_e)^2 over the M lower-triangle elements, Adam
(beta1 0.9, beta2 0.999, eps 1e-8).  Parameters are used rounded to BF16 (round
to nearest, ties to even, applied to their FP32 values).

The densities entering the features, the extrapolation and the target are
Loewdin densities D_L = S^{1/2} D S^{1/2} of their own geometries
(lowdin_factors); the predicted D_L goes back to the AO basis with the new
geometry's S^{-1/2} (apply).
"""
import numpy as np

F = 12


def nparams(H):
    return H * F + 2 * H + 1


def unpack(p, H):
    p = np.asarray(p, dtype=np.float64)
    W1 = p[:H * F].reshape(H, F)
    b1 = p[H * F:H * F + H]
    w2 = p[H * F + H:H * F + 2 * H]
    b2 = p[H * F + 2 * H]
    return W1, b1, w2, b2


def bf16_round(x):
    """FP32 values rounded to BF16 (nearest, ties to even), returned as float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p, X, H):
    W1, b1, w2, b2 = unpack(p, H)
    h = np.tanh(np.asarray(X, dtype=np.float64) @ W1.T + b1)
    return h @ w2 + b2, h


def loss_grad(p, X, t, H):
    """L and dL/dp (params layout) for L = (1/M) sum (y - t)^2."""
    X = np.asarray(X, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    M = X.shape[0]
    W1, b1, w2, b2 = unpack(p, H)
    y, h = forward(p, X, H)
    r = y - t
    g = 2.0 * r / M
    dw2 = h.T @ g
    db2 = g.sum()
    dz = np.outer(g, w2) * (1.0 - h * h)
    dW1 = dz.T @ X
    db1 = dz.sum(axis=0)
    grad = np.concatenate([dW1.ravel(), db1, dw2, [db2]])
    return float(np.mean(r * r)), grad


def adam_step(p, g, m, v, k, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Step k (1-based) of Adam; returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** k)
    vh = v / (1 - b2 ** k)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def extrapolate(D0, D1, D2):
    """Three-point (quadratic) extrapolation of the next density."""
    return 3.0 * D0 - 3.0 * D1 + D2


def lower_index(N):
    """(mu, nu) of the lower-triangle elements in the order e = mu (mu + 1) / 2 + nu."""
    mu, nu = np.tril_indices(N)
    return mu, nu


def _pair_dist(R, A, B):
    R = np.asarray(R, dtype=np.float64).reshape(-1, 3)
    return np.linalg.norm(R[A] - R[B], axis=1)


def scales(D0, D1, S1, S0, R1, R0, ao_atom):
    """Feature scales: RMS over the lower triangle of D_t - D_{t-1},
    S_{t+1} - S_t and r_{t+1} - r_t (r the distance of the two AOs' atoms)."""
    mu, nu = lower_index(D0.shape[0])
    A, B = np.asarray(ao_atom)[mu], np.asarray(ao_atom)[nu]
    rms = lambda v: max(float(np.sqrt(np.mean(v * v))), 1e-12)
    return (rms((D0 - D1)[mu, nu]), rms((S1 - S0)[mu, nu]), rms(_pair_dist(R1, A, B) - _pair_dist(R0, A, B)))


def features(D0, D1, D2, S1, S0, R1, R0, Rm, ao_atom, ao_l, sd=1.0, ss=1.0, sr=1.0):
    """The 12 features of every lower-triangle element and the extrapolation
    D_x: the last three densities, two overlaps and three atom-pair distances
    as scaled differences,
      D_t, (D_t - D_{t-1})/sd, (D_{t-1} - D_{t-2})/sd, (D_t - 2 D_{t-1} + D_{t-2})/sd,
      S_{t+1}, (S_{t+1} - S_t)/ss, r_{t+1}/10, (r_{t+1} - r_t)/sr, (r_t - r_{t-1})/sr,
      same-atom flag, (l_mu + l_nu)/4, |l_mu - l_nu|/4."""
    N = D0.shape[0]
    mu, nu = lower_index(N)
    Dx = extrapolate(D0, D1, D2)
    A, B = np.asarray(ao_atom)[mu], np.asarray(ao_atom)[nu]
    la, lb = np.asarray(ao_l)[mu], np.asarray(ao_l)[nu]
    r1, r0, rm = _pair_dist(R1, A, B), _pair_dist(R0, A, B), _pair_dist(Rm, A, B)
    d0, d1, d2 = D0[mu, nu], D1[mu, nu], D2[mu, nu]
    X = np.stack([d0, (d0 - d1) / sd, (d1 - d2) / sd, (d0 - 2 * d1 + d2) / sd, S1[mu, nu],
                  (S1[mu, nu] - S0[mu, nu]) / ss, 0.1 * r1, (r1 - r0) / sr, (r0 - rm) / sr,
                  (A == B).astype(float), 0.25 * (la + lb), 0.25 * np.abs(la - lb)], axis=1)
    return X, Dx[mu, nu]


def apply(Dx_lower, y, scale, N, S_mhalf=None):
    """Symmetric N x N density from lower-triangle values D_x + scale * y;
    with S_mhalf (the S^{-1/2} of lowdin_factors) the values are Loewdin
    densities and the result is taken back to the AO basis,
    D = S^{-1/2} D_L S^{-1/2}."""
    mu, nu = lower_index(N)
    D = np.zeros((N, N))
    v = Dx_lower + scale * np.asarray(y, dtype=np.float64)
    D[mu, nu] = v
    D[nu, mu] = v
    if S_mhalf is not None:
        D = S_mhalf @ D @ S_mhalf
    return D


def lowdin_factors(S, tau):
    """S^{1/2} over all eigenpairs of the overlap matrix and the pseudo-inverse
    S^{-1/2} over the eigenvalues above tau (the linear-dependence threshold of
    the orthogonaliser).  The guess history holds Loewdin densities
    D_L = S^{1/2} D S^{1/2}: the density in the symmetrically orthonormalised
    basis, idempotent with elements bounded by one, continuous in the nuclear
    positions, so that its extrapolation and the network's correction are not
    dominated by the large, nearly unphysical AO-basis components that an
    almost linearly dependent basis gives D."""
    w, U = np.linalg.eigh(np.asarray(S, dtype=np.float64))
    keep = w > tau
    Sh = (U * np.sqrt(np.clip(w, 0.0, None))) @ U.T
    Smh = (U[:, keep] / np.sqrt(w[keep])) @ U[:, keep].T
    return Sh, Smh
