"""Pins of the learned-guess oracle (oracle/mlp.py) against facts that do not
come from the oracle itself: finite differences of its loss, the BF16 format's
definition, Adam's first step, exactness of quadratic extrapolation, and
hand-built feature values."""
import numpy as np

from oracle import mlp as O


def test_bf16_rounding_definition():
    one = 1.0
    # 8 significant bits: the spacing above 1 is 2^-7
    assert O.bf16_round(one) == 1.0
    assert O.bf16_round(1 + 2.0 ** -8) == 1.0                     # tie -> even (mantissa 0)
    assert O.bf16_round(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6       # tie -> even (mantissa 2)
    assert O.bf16_round(1 + 2.0 ** -8 + 2.0 ** -20) == 1 + 2.0 ** -7
    assert O.bf16_round(-2.5) == -2.5
    x = np.float32(0.1)
    r = O.bf16_round(x)
    assert abs(r - 0.1) <= 2.0 ** -8 * 0.1 and r.dtype == np.float64


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    H, M = 32, 40
    p = rng.normal(scale=0.3, size=O.nparams(H))
    X = rng.normal(size=(M, O.F))
    t = rng.normal(size=M)
    L, g = O.loss_grad(p, X, t, H)
    h = 1e-6
    idx = rng.choice(len(p), size=25, replace=False).tolist() + [len(p) - 1, 0, H * O.F, H * O.F + H]
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (O.loss_grad(pp, X, t, H)[0] - O.loss_grad(pm, X, t, H)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * (1 + abs(fd)), (i, fd, g[i])


def test_forward_closed_form():
    H = 32
    p = np.zeros(O.nparams(H))
    W1, b1, w2, b2 = O.unpack(p, H)
    # b1 = atanh(1/2) makes every hidden unit 1/2 for any input when W1 = 0
    p[H * O.F:H * O.F + H] = np.arctanh(0.5)
    p[H * O.F + H:H * O.F + 2 * H] = np.arange(H)
    p[-1] = 0.25
    y, h = O.forward(p, np.ones((3, O.F)), H)
    assert np.allclose(h, 0.5) and np.allclose(y, 0.5 * np.arange(H).sum() + 0.25)


def test_adam_first_step_is_lr_times_sign():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([3.0, -1e-3, 0.0])
    q, m, v = O.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> step lr * g / (|g| + eps)
    assert np.allclose(q[:2], p[:2] - 0.01 * np.sign(g[:2]), atol=1e-8)
    assert q[2] == p[2]


def test_quadratic_extrapolation_is_exact_for_quadratics():
    rng = np.random.default_rng(1)
    A, B, C = (rng.normal(size=(5, 5)) for _ in range(3))
    D = lambda s: A + B * s + C * s * s
    assert np.allclose(O.extrapolate(D(3), D(2), D(1)), D(4), atol=1e-12)


def test_features_on_a_hand_built_case():
    # two atoms, three AOs: (atom 0, l 0), (atom 0, l 1), (atom 1, l 2)
    N = 3
    D0 = np.arange(9.0).reshape(3, 3)
    D0 = D0 + D0.T
    D1, D2 = 0.5 * D0, 0.25 * D0
    S1, S0 = np.eye(3) * 2, np.eye(3)
    R1 = np.array([[0, 0, 0], [0, 0, 3.0]])
    R0 = np.array([[0, 0, 0], [0, 0, 2.0]])
    Rm = np.array([[0, 0, 0], [0, 0, 1.0]])
    sd, ss, sr = 2.0, 4.0, 0.5
    X, Dx = O.features(D0, D1, D2, S1, S0, R1, R0, Rm, [0, 0, 1], [0, 1, 2], sd, ss, sr)
    mu, nu = O.lower_index(N)
    assert X.shape == (6, O.F)
    assert np.allclose(Dx, (3 - 1.5 + 0.25) * D0[mu, nu])
    e = list(zip(mu, nu)).index((2, 0))     # AO 2 on atom 1, AO 0 on atom 0
    d = D0[2, 0]
    assert np.isclose(X[e, 0], d) and np.isclose(X[e, 1], 0.5 * d / sd) and np.isclose(X[e, 2], 0.25 * d / sd)
    assert np.isclose(X[e, 3], 0.25 * d / sd)
    assert np.isclose(X[e, 6], 0.3) and np.isclose(X[e, 7], 1.0 / sr) and np.isclose(X[e, 8], 1.0 / sr)
    assert X[e, 9] == 0.0 and np.isclose(X[e, 10], 0.5) and np.isclose(X[e, 11], 0.5)
    e = list(zip(mu, nu)).index((1, 0))
    assert X[e, 9] == 1.0 and X[e, 6] == 0.0 and X[e, 7] == 0.0
    e = list(zip(mu, nu)).index((2, 2))
    assert np.isclose(X[e, 4], 2.0) and np.isclose(X[e, 5], 1.0 / ss)
    # scales: RMS over the lower triangle of the first differences
    sd0, ss0, sr0 = O.scales(D0, D1, S1, S0, R1, R0, [0, 0, 1])
    assert np.isclose(sd0, np.sqrt(np.mean((0.5 * D0[mu, nu]) ** 2)))
    assert np.isclose(ss0, np.sqrt(3 / 6)) and np.isclose(sr0, np.sqrt(2 / 6))   # pairs (2,0), (2,1) move


def test_lowdin_factors_square_roots_and_projector():
    """S^{1/2} squares to S, S^{-1/2} inverts it on the kept space; the Loewdin
    density of a closed-shell density is idempotent with eigenvalues 0 and 1;
    the round trip through apply() gives the AO density back.  A dropped
    eigenvalue turns S^{-1/2} S S^{-1/2} into the projector on the kept space."""
    rng = np.random.default_rng(4)
    N, nocc = 7, 3
    G = rng.normal(size=(N, N))
    S = G @ G.T + 0.05 * np.eye(N)
    Sh, Smh = O.lowdin_factors(S, 1e-10)
    assert np.allclose(Sh @ Sh, S, atol=1e-12 * np.abs(S).max())
    assert np.allclose(Smh @ S @ Smh, np.eye(N), atol=1e-10)
    # a closed-shell density: D = C C^T with C^T S C = I
    X = Smh
    C = X @ np.linalg.qr(rng.normal(size=(N, nocc)))[0]
    D = C @ C.T
    DL = Sh @ D @ Sh
    assert np.allclose(DL @ DL, DL, atol=1e-10)
    assert np.allclose(np.sort(np.linalg.eigvalsh(DL)), [0] * (N - nocc) + [1] * nocc, atol=1e-10)
    mu, nu = O.lower_index(N)
    assert np.allclose(O.apply(DL[mu, nu], np.zeros(len(mu)), 1.0, N, Smh), D, atol=1e-10)
    # a near-null direction below the threshold is dropped
    w, U = np.linalg.eigh(S)
    w2 = w.copy()
    w2[0] = 1e-12
    S2 = (U * w2) @ U.T
    _, Smh2 = O.lowdin_factors(S2, 1e-9)
    P = Smh2 @ S2 @ Smh2
    assert np.allclose(P, np.eye(N) - np.outer(U[:, 0], U[:, 0]), atol=1e-8)
