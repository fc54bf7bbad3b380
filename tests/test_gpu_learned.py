"""The learned coefficient predictor on the GPU against the oracle (oracle/mlp.py).

Tolerances:
* initial weights: bit-exact (integer SplitMix64 counters, one FP64 affine map,
  one rounding to FP32 on both sides);
* sample (features, target, W1^T W1, ||S b||): FP64 on both sides up to the
  least-squares solve (relative 1e-10 on a well-conditioned history), then one
  rounding to FP32: relative 1e-6;
* loss and gradients: FP32 arithmetic with bfloat16 weights on both sides (the
  same rounded weights), different summation orders over K <= 256 terms:
  relative 1e-3 of each tensor's largest entry;
* selection: the decision rule (network residual <= 1.5 x least squares) is
  taken by the oracle in FP64 from the same FP32 prediction; cases within
  1e-6 of the threshold would be skipped (none occur with these seeds).
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import krylov, method, mlp as omlp, sketch

pytestmark = pytest.mark.gpu

DEV = "cuda"
M, S_ROWS, SEED = 6, 40, 0x5EEDBA5E


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_02156_gb300 as sa
    sa.load()
    yield


def _sa():
    import paper_2309_02156_gb300 as sa
    return sa


def _tensor(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device=DEV, dtype=dtype)


def _split(net, flat):
    inp, hid, out = net.inp, net.hidden, net.M
    sizes = [hid * inp, hid, hid * hid, hid, out * hid, out]
    parts, o = [], 0
    for k in sizes:
        parts.append(flat[o:o + k])
        o += k
    assert o == flat.size
    return [parts[0].reshape(hid, inp), parts[1], parts[2].reshape(hid, hid), parts[3],
            parts[4].reshape(out, hid), parts[5]]


def _oracle_params(net, flat, norm):
    W1, b1, W2, b2, W3, b3 = _split(net, flat)
    inp = net.inp
    return omlp.Params(W1, b1, W2, b2, W3, b3, norm[:inp], norm[inp:2 * inp], norm[2 * inp:])


@pytest.mark.parametrize("Mq,s,hid,seed", [(20, 80, 256, 1), (6, 40, 48, 0xC0FFEE)])
def test_init_matches_oracle(Mq, s, hid, seed):
    net = _sa().MLP(Mq, s, hidden=hid, max_batch=8, seed=seed)
    flat, norm = net.get_params()
    W1, b1, W2, b2, W3, b3 = _split(net, flat)
    inp = 4 * Mq + s
    assert np.array_equal(W1, omlp.he_uniform(seed, hid, inp, 0))
    assert np.array_equal(W2, omlp.he_uniform(seed, hid, hid, hid * inp))
    assert np.array_equal(W3, omlp.he_uniform(seed, Mq, hid, hid * inp + hid * hid))
    assert not b1.any() and not b2.any() and not b3.any()
    assert np.array_equal(norm, np.r_[np.zeros(inp), np.ones(inp), np.ones(Mq)].astype(np.float32))
    net.close()


def _synthetic_samples(rng, Mq, s, B):
    inp = 4 * Mq + s
    F = rng.standard_normal((B, inp))
    T = F[:, :Mq] + 0.3 * rng.standard_normal((B, Mq))
    W1 = rng.standard_normal((B, s, Mq))
    G = np.einsum("bqi,bqj->bij", W1, W1)
    nb = 1.0 + rng.random(B) * 3
    S = np.concatenate([F, T, G.reshape(B, -1), nb[:, None]], axis=1).astype(np.float32)
    return S


@pytest.mark.parametrize("Mq,s,hid,B", [(20, 80, 256, 64), (6, 40, 48, 37), (3, 16, 20, 1)])
def test_loss_and_gradients_match_oracle(Mq, s, hid, B):
    rng = np.random.default_rng(Mq * 1000 + B)
    net = _sa().MLP(Mq, s, hidden=hid, max_batch=B, seed=5)
    flat, _ = net.get_params()
    inp = 4 * Mq + s
    flat = flat.copy()
    o_b1 = hid * inp
    flat[o_b1:o_b1 + hid] = 0.1 * rng.standard_normal(hid)                      # nonzero biases
    o_b2 = o_b1 + hid + hid * hid
    flat[o_b2:o_b2 + hid] = 0.1 * rng.standard_normal(hid)
    flat[-Mq:] = 0.1 * rng.standard_normal(Mq)
    norm = np.r_[rng.standard_normal(inp) * 0.1, 1 + rng.random(inp), 0.5 + rng.random(Mq)]
    norm = norm.astype(np.float32)
    net.set_params(flat, norm)
    S = _synthetic_samples(rng, Mq, s, B)
    loss, g = net.loss_grad(_tensor(S, torch.float32))
    p = _oracle_params(net, flat, norm)
    F, T = S[:, :inp], S[:, inp:inp + Mq]
    G = S[:, inp + Mq:inp + Mq + Mq * Mq].reshape(B, Mq, Mq)
    nb = S[:, -1]
    l_ref, g_ref = omlp.loss_and_grad(p, F, T, G, nb, dtype=np.float32, round_bf16=True)
    assert loss == pytest.approx(l_ref, rel=1e-4)
    for got, ref in zip(_split(net, g), g_ref):
        assert np.abs(got - ref).max() <= 1e-3 * np.abs(ref).max() + 1e-12
    # prediction equals the forward pass
    y = net.predict(_tensor(S, torch.float32)).cpu().numpy()
    y_ref, _ = omlp.forward(p, F, dtype=np.float32, round_bf16=True)
    assert np.abs(y - y_ref).max() <= 1e-4 * (np.abs(y_ref).max() + 1)
    net.close()


def test_adam_step_matches_oracle():
    rng = np.random.default_rng(11)
    Mq, s, hid, B = 6, 40, 48, 32
    net = _sa().MLP(Mq, s, hidden=hid, max_batch=B, seed=9)
    flat0, norm = net.get_params()
    S = _synthetic_samples(rng, Mq, s, B)
    St = _tensor(S, torch.float32)
    _, g = net.loss_grad(St)
    losses = net.train(St, epochs=1, batch=B, lr=1e-3, seed=3)
    flat1, _ = net.get_params()
    # oracle Adam on the GPU gradient of the same batch (the batch mean does not
    # depend on the shuffle beyond rounding)
    p = [a.copy() for a in _split(net, flat0)]
    gs = _split(net, g)
    m = [np.zeros_like(a) for a in p]
    v = [np.zeros_like(a) for a in p]
    omlp.adam_update(p, gs, m, v, 1, lr=1e-3)
    ref = np.concatenate([a.ravel() for a in p])
    big = np.abs(g) > 1e-3 * np.abs(g).max()          # sign(g) decides the first step
    assert np.abs(flat1 - ref)[big].max() <= 1e-6
    assert np.abs(flat1 - flat0).max() <= 1e-3 * (1 + 1e-5)
    assert losses.shape == (1,) and np.isfinite(losses[0])
    net.close()


def _gaussian_sequence(p, steps, seed):
    """A history of random Gaussian columns (well-conditioned least squares)."""
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(p.n) for _ in range(M + steps)]


def test_sample_matches_oracle_features():
    p = workloads.plain_nonsym(24)
    cols = _gaussian_sequence(p, 9, 4)
    seq = _sa().Sequence(p.n, M, S_ROWS, zeta=8, seed=SEED)
    S = sketch.sparse_sign_matrix(p.n, S_ROWS, 8, SEED)
    inp = 4 * M + S_ROWS
    stride = inp + M + M * M + 1
    buf = torch.empty(stride, dtype=torch.float32, device=DEV)
    ys, checked = [], 0
    for c in cols[:M]:
        seq.push(_tensor(c))
    for k in range(9):
        i = 3 + k
        rowptr, colind, vals, b = workloads.csr_system(p, i)
        A = _sa().CSR(_tensor(rowptr, torch.int32), _tensor(colind, torch.int32), _tensor(vals))
        x0 = torch.empty(p.n, dtype=torch.float64, device=DEV)
        seq.guess(A, _tensor(b), x0)
        X = np.stack(cols[k:k + M], axis=1)
        ref = method.sketched_guess(krylov.csr(rowptr, colind, vals, p.n), b, X, S)
        if len(ys) >= 4:
            seq.last_sample(buf)
            got = buf.cpu().numpy().astype(np.float64)
            feat = omlp.features(ref.W, M, [ys[-1], ys[-2], ys[-3], ys[-4]])
            W1, wb = ref.W[:, :M], ref.W[:, M]
            want = np.r_[feat, ref.y, (W1.T @ W1).ravel(), np.linalg.norm(wb)]
            np.testing.assert_allclose(got, want, rtol=2e-6, atol=2e-6 * np.abs(want[:inp]).max())
            checked += 1
        else:
            with pytest.raises(_sa().SeqError):
                seq.last_sample(buf)
        ys.append(ref.y)
        seq.push(_tensor(cols[k + M]))
    assert checked == 5
    seq.close()


def test_learned_selection_and_fallback():
    """A network whose output is the least-squares y (rounded to FP32) is used;
    one whose output is far from it falls back to least squares."""
    p = workloads.plain_nonsym(24)
    cols = _gaussian_sequence(p, 8, 8)
    seq = _sa().Sequence(p.n, M, S_ROWS, zeta=8, seed=SEED, guess="learned")
    net = _sa().MLP(M, S_ROWS, hidden=16, max_batch=4, seed=2)
    flat, norm = net.get_params()
    flat = flat.copy()
    o_W3 = net.nparams - M - M * net.hidden
    flat[o_W3:o_W3 + M * net.hidden] = 0.0
    seq.set_learned(net)
    S = sketch.sparse_sign_matrix(p.n, S_ROWS, 8, SEED)
    ys, outcomes = [], []
    for c in cols[:M]:
        seq.push(_tensor(c))
    for k in range(8):
        i = 2 + k
        rowptr, colind, vals, b = workloads.csr_system(p, i)
        A_ref = krylov.csr(rowptr, colind, vals, p.n)
        X = np.stack(cols[k:k + M], axis=1)
        ref = method.sketched_guess(A_ref, b, X, S)
        base = np.zeros(M, np.float32)
        if ys:
            base[:M - 1] = ys[-1][1:].astype(np.float32)
        want_net = k % 2 == 0
        if want_net:
            b3 = (ref.y.astype(np.float32) - base).astype(np.float32)
        else:                                   # far from the least-squares y
            b3 = np.full(M, 50.0 * max(1.0, np.abs(ref.y).max()), np.float32)
        flat[-M:] = b3
        net.set_params(flat, norm)
        A = _sa().CSR(_tensor(rowptr, torch.int32), _tensor(colind, torch.int32), _tensor(vals))
        x0 = torch.empty(p.n, dtype=torch.float64, device=DEV)
        info = seq.guess(A, _tensor(b), x0)
        x0 = x0.cpu().numpy()
        if len(ys) >= 4:
            yhat = (base + b3).astype(np.float32).astype(np.float64)
            rho_net = np.linalg.norm(ref.W[:, :M] @ yhat - ref.W[:, M])
            use = rho_net <= 1.5 * ref.rho_s
            assert abs(rho_net / (1.5 * ref.rho_s) - 1) > 1e-6
            assert use == want_net
            assert info["fallback"] == (not use)
            assert info["net_resid"] == pytest.approx(rho_net, rel=1e-6)
            x_want = X @ yhat if use else ref.x0
            assert np.linalg.norm(x0 - x_want) <= 1e-6 * np.linalg.norm(x_want)
            assert info["guess_relres"] == pytest.approx(method.relres(A_ref, b, x_want), rel=1e-5)
            outcomes.append(use)
        else:
            assert not info["fallback"] and info["net_resid"] == -1.0
            assert np.linalg.norm(x0 - ref.x0) <= 1e-10 * np.linalg.norm(ref.x0)
        ys.append(ref.y)
        seq.push(_tensor(cols[k + M]))
    assert True in outcomes and False in outcomes
    seq.close()
    net.close()


def test_training_is_deterministic_and_reduces_loss():
    """Samples from a smooth solution sequence (GPU solves, FP64 GMRES to 1e-10):
    training lowers the excess-residual loss and repeats bit for bit."""
    p = workloads.plain_nonsym(24)
    seq = _sa().Sequence(p.n, M, S_ROWS, zeta=8, seed=SEED, krylov="gmres")
    inp = 4 * M + S_ROWS
    stride = inp + M + M * M + 1
    samples = []
    for i in range(60):
        rowptr, colind, vals, b = workloads.csr_system(p, i)
        A = _sa().CSR(_tensor(rowptr, torch.int32), _tensor(colind, torch.int32), _tensor(vals))
        x = torch.empty(p.n, dtype=torch.float64, device=DEV)
        seq.guess(A, _tensor(b), x)
        if i >= M + 4:
            buf = torch.empty(stride, dtype=torch.float32, device=DEV)
            seq.last_sample(buf)
            samples.append(buf)
        info = seq.solve(A, _tensor(b), 1e-10, x)
        assert info["status"] == 0
        seq.push(x)
    St = torch.stack(samples)
    assert torch.isfinite(St).all()
    results = []
    for _ in range(2):
        net = _sa().MLP(M, S_ROWS, hidden=64, max_batch=16, seed=4)
        net.fit_normalization(St)
        l0, _ = net.loss_grad(St[:16])
        losses = net.train(St, epochs=40, batch=16, lr=1e-3, seed=6)
        l1, _ = net.loss_grad(St[:16])
        results.append((net.get_params()[0], losses, l0, l1))
        net.close()
    (pa, la, l0, l1), (pb, lb, _, _) = results
    assert np.array_equal(pa, pb) and np.array_equal(la, lb)
    assert l1 < 0.5 * l0 and la[-1] < la[0]
    seq.close()


def test_learned_gain_over_least_squares():
    """What the trained network gains: two contexts see identical histories
    (the least-squares path's solutions are pushed into both); the network is
    trained on the first 40 systems' samples and used on the next 15.  The
    fallback bounds the loss (a rejected prediction leaves the least-squares
    guess, so the solve is the same); the gain is reported, not assumed."""
    p = workloads.plain_nonsym(48)
    mk = lambda: _sa().Sequence(p.n, M, S_ROWS, zeta=8, seed=SEED, guess="learned", krylov="gmres")
    c_ls, c_net = mk(), mk()
    inp = 4 * M + S_ROWS
    stride = inp + M + M * M + 1
    samples = []
    x = torch.empty(p.n, dtype=torch.float64, device=DEV)
    y = torch.empty(p.n, dtype=torch.float64, device=DEV)

    def system(i):
        rowptr, colind, vals, b = workloads.csr_system(p, i)
        return _sa().CSR(_tensor(rowptr, torch.int32), _tensor(colind, torch.int32), _tensor(vals)), _tensor(b)

    for i in range(40):
        A, b = system(i)
        c_ls.guess(A, b, x)
        c_net.guess(A, b, y)
        if i >= M + 4:
            buf = torch.empty(stride, dtype=torch.float32, device=DEV)
            c_ls.last_sample(buf)
            samples.append(buf)
        assert c_ls.solve(A, b, 1e-10, x)["status"] == 0
        c_ls.push(x)
        c_net.push(x)
    net = _sa().MLP(M, S_ROWS, hidden=64, max_batch=16, seed=3)
    St = torch.stack(samples)
    net.fit_normalization(St)
    net.train(St, epochs=60, batch=16, lr=1e-3, seed=1)
    c_net.set_learned(net)
    it_ls, it_net, used = [], [], []
    for i in range(40, 55):
        A, b = system(i)
        g1 = c_ls.guess(A, b, x)
        g2 = c_net.guess(A, b, y)
        i1 = c_ls.solve(A, b, 1e-10, x)
        i2 = c_net.solve(A, b, 1e-10, y)
        assert i1["status"] == 0 and i2["status"] == 0
        it_ls.append(i1["iters"])
        it_net.append(i2["iters"])
        used.append(not g2["fallback"])
        if g2["fallback"]:
            assert g2["guess_relres"] == pytest.approx(g1["guess_relres"], rel=1e-12)
            assert i2["iters"] == i1["iters"]
        else:
            assert g2["sketch_resid"] <= 1.5 * g1["sketch_resid"] * (1 + 1e-12)
        c_ls.push(x)
        c_net.push(x)
    gain = np.mean(it_ls) - np.mean(it_net)
    print(f"learned form: network used on {sum(used)}/{len(used)} systems, mean GMRES iterations "
          f"{np.mean(it_net):.1f} vs {np.mean(it_ls):.1f} with least squares (gain {gain:+.1f})")
    assert np.mean(it_net) <= 1.1 * np.mean(it_ls) + 2
    c_ls.close()
    c_net.close()
    net.close()


def test_context_learned_train_save_load():
    """seq_learned_train on a context without a predictor equals
    seq_mlp_create(M, s, 256, 32, seed) + seq_mlp_fit_normalization +
    seq_mlp_train(epochs, 32, 1e-3, seed), bit for bit; seq_learned_save and
    seq_learned_load carry the trained network into a second context, whose
    parameters and learned-mode guesses then equal the first's."""
    sa = _sa()
    Mq, s, count, epochs, seed = 6, 40, 80, 3, 0xA11CE
    rng = np.random.default_rng(17)
    samples = _tensor(_synthetic_samples(rng, Mq, s, count), torch.float32)
    n = 64
    ctx = sa.Sequence(n, Mq, s, zeta=8, seed=SEED, guess="learned")
    ctx.learned_train(samples, epochs, seed)
    blob = ctx.learned_save()
    ref = sa.MLP(Mq, s, hidden=256, max_batch=32, seed=seed)
    ref.fit_normalization(samples)
    ref.train(samples, epochs=epochs, batch=32, lr=1e-3, seed=seed)
    p_ref, n_ref = ref.get_params()
    hdr = np.frombuffer(blob[:16], dtype=np.int32)
    assert list(hdr) == [0x4C514553, Mq, s, 256]
    body = np.frombuffer(blob[16:], dtype=np.float32)
    assert body.size == p_ref.size + n_ref.size
    assert np.array_equal(body[:p_ref.size], p_ref)          # bit for bit
    assert np.array_equal(body[p_ref.size:], n_ref)
    # Load into a second context and read it back.
    ctx2 = sa.Sequence(n, Mq, s, zeta=8, seed=SEED, guess="learned")
    ctx2.learned_load(blob)
    assert ctx2.learned_save() == blob
    # A header for another history length is rejected.
    bad = bytearray(blob)
    bad[4:8] = np.int32(Mq + 1).tobytes()
    with pytest.raises(sa.SeqError) as e:
        ctx2.learned_load(bytes(bad))
    assert e.value.code == -1
    with pytest.raises(sa.SeqError):
        ctx2.learned_load(blob[:-4])
    # Both contexts guess the same from the same history with the loaded net.
    p = workloads.plain_nonsym(8)
    guesses = []
    for c in (ctx, ctx2):
        hist_rng = np.random.default_rng(3)
        outs = []
        for i in range(Mq + 6):
            rowptr, colind, vals, b = workloads.csr_system(p, i)
            A = sa.CSR(_tensor(rowptr, torch.int32), _tensor(colind, torch.int32), _tensor(vals))
            x = torch.empty(n, dtype=torch.float64, device=DEV)
            g = c.guess(A, _tensor(b), x)
            outs.append((x.cpu().numpy(), g["net_resid"]))
            c.push(_tensor(hist_rng.standard_normal(n)))
        guesses.append(outs)
    for (x1, r1), (x2, r2) in zip(*guesses):
        assert np.array_equal(x1, x2) and r1 == r2
    assert any(r > 0 for _, r in guesses[0])                 # the network was consulted
    ref.close()
    ctx.close()
    ctx2.close()
