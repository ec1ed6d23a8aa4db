"""Learned SCF guess on the GPU against the CPU oracle (oracle/mlp.py):
the BF16 network kernels (forward, backward, Adam), the feature pipeline and
the extrapolated / learned guess densities inside a context, training, and the
invariance of the converged answer to the guess.

Tolerances: the kernels accumulate in FP32 with the same BF16-rounded weights
as the oracle, so forward values agree to ~1e-5 relative and gradients to
~1e-4 of their largest entry (FP32 sums over M elements in a different order)."""
import dataclasses

import numpy as np
import pytest

from oracle import mlp as O
from paper_2407_19614_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _R():
    from paper_2407_19614_gb300 import rihf as R
    R.load()
    return R


def _rand_net(H, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return (rng.normal(scale=scale, size=O.nparams(H))).astype(np.float32)


@pytest.mark.parametrize("H,M", [(256, 1000), (64, 37), (512, 300)])
def test_mlp_kernels_against_oracle(H, M):
    R = _R()
    rng = np.random.default_rng(H + M)
    p = _rand_net(H, H)
    X = rng.normal(size=(M, O.F)).astype(np.float32)
    t = rng.normal(size=M).astype(np.float32)
    out = R.mlp_eval(p, X, t, lr=1e-3, iters=1, hidden=H)
    pb = O.bf16_round(p)
    y_o, _ = O.forward(pb, X.astype(np.float64), H)
    L_o, g_o = O.loss_grad(pb, X.astype(np.float64), t.astype(np.float64), H)
    assert np.abs(out["y"] - y_o).max() <= 2e-5 * (1 + np.abs(y_o).max())
    assert abs(out["loss2"][0] / M - L_o) <= 1e-5 * L_o
    assert abs(out["loss2"][1] - np.sum(t.astype(np.float64) ** 2)) <= 1e-5 * np.sum(t ** 2)
    gmax = np.abs(g_o).max()
    assert np.abs(out["grad"] - g_o).max() <= 1e-4 * gmax
    # one Adam step from zero moments on the FP32 master parameters
    q_o, _, _ = O.adam_step(p.astype(np.float64), g_o, 0.0, 0.0, 1, lr=1e-3)
    big = np.abs(g_o) > 1e-3 * gmax
    assert np.abs(out["params"] - q_o)[big].max() <= 1e-5
    assert np.abs(out["params"] - p).max() <= 1e-3 * 1.0001


def test_mlp_training_reduces_loss_and_follows_oracle():
    R = _R()
    H, M = 64, 2000
    rng = np.random.default_rng(5)
    X = rng.normal(size=(M, O.F)).astype(np.float32)
    t = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - 0.3 * np.tanh(X[:, 3])).astype(np.float32)
    p = _rand_net(H, 9, scale=0.2)
    lr, K = 3e-3, 300
    out = R.mlp_eval(p, X, t, lr=lr, iters=K, hidden=H)
    losses = out["losses"] / M
    assert losses[-1] < 0.2 * losses[0]
    # the first steps against the oracle's Adam with BF16-rounded weights
    q, m, v = p.astype(np.float64), 0.0, 0.0
    for k in range(1, 6):
        L, g = O.loss_grad(O.bf16_round(q.astype(np.float32)), X, t, H)
        assert abs(losses[k - 1] - L) <= 2e-4 * L, (k, losses[k - 1], L)
        q, m, v = O.adam_step(q, g, m, v, k, lr=lr)
        q = q.astype(np.float32).astype(np.float64)


def _trajectory(mol, steps, seed=0):
    """Velocity-Verlet geometries from an FP64 context (previous-orbital guess)."""
    R = _R()
    ctx = R.Context(mol, conv_e=1e-9, conv_diis=1e-8, max_iter=80)
    m = W.masses_au(mol.Z)[:, None]
    x = mol.xyz.copy()
    v = W.maxwell_boltzmann(mol.Z, 300.0, seed)
    dt = 0.5 * W.FS_TO_AU
    ctx.scf(guess=0, outputs=False)
    g = ctx.gradient()
    xs = []
    for _ in range(steps):
        a = -g / m
        x = x + v * dt + 0.5 * a * dt * dt
        xs.append(x.copy())
        ctx.update_geometry(x)
        ctx.scf(guess=2, outputs=False)
        gn = ctx.gradient()
        v = v + 0.5 * (a - gn / m) * dt
        g = gn
    return [mol.xyz.copy()] + xs


def _ao_maps(mol, pure=True):
    ao_atom, ao_l = [], []
    for sh in mol.primary:
        nf = 2 * sh.l + 1 if pure else (sh.l + 1) * (sh.l + 2) // 2
        ao_atom += [sh.atom] * nf
        ao_l += [sh.l] * nf
    return np.array(ao_atom), np.array(ao_l)


def test_extrapolated_and_learned_guess_pipeline_against_oracle():
    R = _R()
    mol = W.water_n(2, 0)
    xs = _trajectory(mol, 6)
    ctx = R.Context(mol, conv_e=1e-10, conv_diis=1e-9, max_iter=80)
    ctx.learn_config(hidden=64, train_steps=100, adam_iters=2, lr=1e-3, seed=3)
    ao_atom, ao_l = _ao_maps(mol)
    Ds, Ss = [], []
    scales = None
    for k, x in enumerate(xs):
        if k:
            ctx.update_geometry(x)
        S1 = ctx.matrix("S")
        params = ctx.learn_params()
        scale = ctx.learn_stats()["scale"]
        out = ctx.scf(guess=4 if k else 0)
        st = ctx.learn_stats()
        Sh, Smh = O.lowdin_factors(S1, 1e-8)       # the context's lindep_tau
        if k >= 3:
            # the history is full: the guess is the extrapolation of the last
            # three converged (Loewdin) densities, plus the network's
            # correction once it has earned its use (guess kind 4), taken
            # back to the AO basis with this geometry's S^{-1/2}
            assert st["last_guess"] in (3, 4)
            assert k >= 6 or st["last_guess"] == 3      # three training examples first
            Dx = Smh @ O.extrapolate(Ds[-1], Ds[-2], Ds[-3]) @ Smh
            if scales is None:
                scales = O.scales(Ds[-1], Ds[-2], S1, Ss[-1], x, xs[k - 1], ao_atom)
            Xo, Dxl = O.features(Ds[-1], Ds[-2], Ds[-3], S1, Ss[-1], x, xs[k - 1], xs[k - 2], ao_atom, ao_l,
                                 *scales)
            Xg = ctx.matrix("FEATURES")
            assert np.abs(Xg - Xo).max() <= 1e-5 * (1 + np.abs(Xo).max())
            Dp = ctx.matrix("DPRED")
            # the AO prediction, and the same in the Loewdin representation
            # (S^{1/2} Dp S^{1/2}: nothing is dropped at this threshold), where
            # the network's FP32 error is not magnified by S^{-1/2}
            DLp = Sh @ Dp @ Sh
            if st["last_guess"] == 3:
                assert np.abs(Dp - Dx).max() <= 1e-9 * (1 + np.abs(Dx).max())
                DLx = O.extrapolate(Ds[-1], Ds[-2], Ds[-3])
                assert np.abs(DLp - DLx).max() <= 1e-10 * (1 + np.abs(DLx).max())
            else:
                y, _ = O.forward(O.bf16_round(params), Xg, 64)
                DLref = O.apply(Dxl, y, scale, Dx.shape[0])
                assert np.abs(DLp - DLref).max() <= 1e-5 * scale * (1 + np.abs(y).max()) + 1e-10
            assert st["trained_steps"] == k - 2
        Ds.append(Sh @ out["D"] @ Sh)
        Ss.append(S1)


def _relaxed(mol, R, gtol=2e-5, iters=400):
    """The molecule's nearest minimum in this basis (steepest descent with a
    step that grows after each accepted step and halves after a rejected one),
    so that a 300 K trajectory from it is a thermal vibration, not the
    relaxation of the generator's strained geometry."""
    ctx = R.Context(mol, conv_e=1e-11, conv_diis=1e-10, max_iter=100)
    x = mol.xyz.copy()
    E = ctx.scf(guess=0, outputs=False)["energy"]
    g = ctx.gradient()
    step = 0.3
    for _ in range(iters):
        if np.abs(g).max() < gtol:
            break
        xn = x - step * g
        ctx.update_geometry(xn)
        En = ctx.scf(guess=2, outputs=False)["energy"]
        if En < E:
            x, E, g = xn, En, ctx.gradient()
            step *= 1.2
        else:
            ctx.update_geometry(x)
            ctx.scf(guess=2, outputs=False)
            step *= 0.5
    ctx.close()
    assert np.abs(g).max() < gtol
    return dataclasses.replace(mol, xyz=x)


def test_learned_guess_keeps_the_answer_and_reports_its_gain():
    """What the trained network gains over the extrapolated guess alone.

    A 300 K trajectory of the water monomer from its relaxed geometry (a
    thermal vibration: the generator's strained geometries make every step a
    large-amplitude jump that no history predicts), replayed by two contexts:
    the extrapolated guess (3) and the learned guess (4), network trained
    online on the first 150 steps, then frozen.  Over the 90 steps after
    training: the network is in use, its out-of-sample error is well below
    the extrapolation's, the SCF needs fewer iterations than from the
    extrapolation alone, and the converged energies agree at every step --
    the guess changes the iteration count, never the answer."""
    R = _R()
    mol = _relaxed(W.water_monomer(0), R)
    xs = _trajectory(mol, 240)
    train = 150
    res = {}
    for guess in (3, 4):
        ctx = R.Context(mol, conv_e=1e-10, conv_diis=1e-9, max_iter=80)
        ctx.learn_config(hidden=256, train_steps=train, adam_iters=4, lr=1e-3, seed=1)
        E, its, ratios, used = [], [], [], []
        for k, x in enumerate(xs):
            if k:
                ctx.update_geometry(x)
            out = ctx.scf(guess=guess if k else 0, outputs=False)
            E.append(out["energy"])
            its.append(out["iterations"])
            st = ctx.learn_stats()
            ratios.append(st["last_ratio"])
            used.append(st["last_guess"] == 4)
        res[guess] = (np.array(E), np.array(its), ratios, used)
        ctx.close()
    E3, i3 = res[3][0], res[3][1]
    E4, i4, ratios, used = res[4]
    assert np.abs(E3 - E4).max() <= 2e-9
    after = slice(train + 4, len(xs))          # steps after the last training example
    finite = [r for r in ratios[:train + 4] if r < 1e299]
    print("\nrelaxed monomer, 300 K: SCF iterations per step over the %d steps after training: "
          "extrapolated %.2f, learned %.2f (network used on %d of them); median out-of-sample error "
          "ratio over the last 20 training steps %.3f" % (len(xs) - after.start, i3[after].mean(), i4[after].mean(),
                                                           sum(used[after]), float(np.median(finite[-20:]))))
    assert all(used[after])
    assert float(np.median(finite[-20:])) < 0.5
    assert i4[after].sum() < i3[after].sum()
