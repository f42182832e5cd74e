"""The BF16 tensor-core MLP kernels against the float64 MLP oracle (same
bfloat16 roundings), and training progress."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1607_05535_gb300 as thor
from oracle import mlp as om

SIZES = [320, 256, 256, 256, 160]

# Both sides round the same values to bfloat16 (inputs, weights, hidden
# activations, the back-propagated gradient). They still differ in two ways:
# (1) where a float32 accumulation and a float64 one fall on opposite sides
# of a bfloat16 rounding boundary, that element moves by one bfloat16 spacing
# (2^-8 relative), a small error; (2) where a hidden pre-activation lies
# within the float32 error of zero, the ReLU masks can disagree and a whole
# gradient element appears on one side only (one such row gives about 5e-3
# relative error in every lower layer's gradients). Rows whose masks a
# float32 error estimate cannot decide are left out of the batch on both
# sides (_decided_rows), and what remains is held to GATE.
GATE = 1e-3
U32 = 2.0 ** -24


def _decided_rows(params, x):
    """Rows of x whose every hidden ReLU mask a float32 evaluation decides
    like the float64 one. Per layer the float32 error of z is estimated as
    4 u K rms_j(h_j W_jn) (about six standard deviations of the rounding
    errors of a K-term float32 sum; products of bfloat16 values are exact in
    float32; the worst-case bound K u sum|h_j W_jn| is some 100 times larger
    and would leave no row decided) plus sum_j d_j |W_jn|, where d_j is one
    bfloat16 spacing for an input that lies within its own layer's estimate
    of a bfloat16 rounding boundary (it may round the other way), else
    zero. A row is kept if every hidden |z| exceeds its estimate."""
    hin = om.bf16(np.asarray(x, dtype=np.float64))
    d = np.zeros_like(hin)
    keep = np.ones(hin.shape[0], dtype=bool)
    for l, (W, b) in enumerate(params[:-1]):
        Wq = om.bf16(W)
        z = hin @ Wq + b
        K = hin.shape[1]
        dz = 4.0 * U32 * K * np.sqrt((hin ** 2) @ (Wq ** 2) / K) + d @ np.abs(Wq) + U32 * np.abs(z)
        keep &= np.all(np.abs(z) > dz, axis=1)
        v = np.maximum(z, 0.0)
        r = om.bf16(v)
        e = np.floor(np.log2(np.maximum(r, 1e-30)))
        s_up = 2.0 ** (e - 7)
        s_dn = np.where(r == 2.0 ** e, s_up / 2, s_up)
        dist = np.minimum(r + s_up / 2 - v, v - (r - s_dn / 2))
        d = np.where((v > 0) & (dist <= dz), s_up, 0.0)
        hin = r
    return keep


def _flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params]).astype(np.float32)


def _unflat(v, sizes):
    out, o = [], 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = v[o:o + a * b].reshape(a, b); o += a * b
        bb = v[o:o + b]; o += b
        out.append((W.astype(np.float64), bb.astype(np.float64)))
    return out


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("m", [64, 200, 1000])
def test_forward_and_gradients_match_oracle(m):
    rng = np.random.default_rng(3)
    params = om.init_params(SIZES, rng)
    params = [(W, 0.05 * rng.standard_normal(W.shape[1])) for W, _ in params]
    flat = _flat(params)
    params32 = _unflat(flat, SIZES)          # exactly what the GPU holds
    x = rng.standard_normal((m, SIZES[0])).astype(np.float32)
    dy = rng.standard_normal((m, SIZES[-1])).astype(np.float32)
    keep = _decided_rows(params32, x)
    assert keep.sum() >= m // 2, keep.sum()
    x, dy, m = x[keep], dy[keep], int(keep.sum())
    net = thor.thor_mlp_create(SIZES, 1024, seed=1)
    try:
        thor.thor_mlp_set_params(net, flat)
        xd = torch.tensor(x, device="cuda")
        yd = torch.empty((m, SIZES[-1]), dtype=torch.float32, device="cuda")
        thor.thor_mlp_forward(net, xd, yd)
        gd = torch.empty(flat.size, dtype=torch.float32, device="cuda")
        thor.thor_mlp_backward(net, torch.tensor(dy, device="cuda"), gd)
        torch.cuda.synchronize()
        y_ref, cache = om.forward(params32, x.astype(np.float64))
        grads = om.backward(params32, cache, dy.astype(np.float64))
        g = _unflat(gd.cpu().numpy(), SIZES)
        errs = [_rel(yd.cpu().numpy(), y_ref)]
        for (gW, gb), (rW, rb) in zip(g, grads):
            errs += [_rel(gW, rW), _rel(gb, rb)]
        print("MLP rows kept %d; rel errors (y, then dW, db per layer):" % m, ["%.2e" % e for e in errs])
        assert max(errs) < GATE, errs
    finally:
        thor.thor_mlp_destroy(net)


def test_training_reduces_loss():
    """Fit a fixed random smooth target; the GPU Adam steps lower the loss."""
    rng = np.random.default_rng(4)
    m = 1024
    x = rng.standard_normal((m, SIZES[0])).astype(np.float32)
    A = rng.standard_normal((SIZES[0], SIZES[-1])).astype(np.float32) / np.sqrt(SIZES[0])
    t = np.tanh(x @ A).astype(np.float32)
    net = thor.thor_mlp_create(SIZES, m, seed=7)
    try:
        xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        losses = []
        for it in range(300):
            thor.thor_mlp_train_step(net, xd, td, 1e-3, loss)
            if it % 50 == 0 or it == 299:
                torch.cuda.synchronize()
                losses.append(float(loss.item()))
        assert losses[-1] < 0.2 * losses[0], losses
    finally:
        thor.thor_mlp_destroy(net)


def test_train_step_matches_oracle_adam():
    """One GPU training step equals the oracle's MSE gradient + Adam step on
    the same bf16-rounded network (float32 vs float64 arithmetic)."""
    rng = np.random.default_rng(5)
    sizes = [40, 64, 16]
    params = om.init_params(sizes, rng)
    flat = _flat(params)
    p32 = _unflat(flat, sizes)
    m = 96
    x = rng.standard_normal((m, sizes[0])).astype(np.float32)
    t = rng.standard_normal((m, sizes[-1])).astype(np.float32)
    net = thor.thor_mlp_create(sizes, 128, seed=0)
    try:
        thor.thor_mlp_set_params(net, flat)
        thor.thor_mlp_train_step(net, torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"), 1e-2)
        new = thor.thor_mlp_get_params(net)
        y, cache = om.forward(p32, x.astype(np.float64))
        grads = om.backward(p32, cache, om.mse_grad(y, t))
        state = [(np.zeros_like(W), np.zeros_like(W), np.zeros_like(b), np.zeros_like(b)) for W, b in p32]
        ref = _flat(om.adam(p32, grads, state, 1e-2, 1))
        # a first Adam step moves each parameter by about lr * sign(g): compare the moves
        move, ref_move = new - flat, ref - flat
        agree = np.mean(np.sign(move) == np.sign(ref_move))
        assert agree > 0.97, agree
        assert np.allclose(np.abs(move[np.abs(ref_move) > 5e-3]), 1e-2, rtol=0.05)
    finally:
        thor.thor_mlp_destroy(net)


@pytest.mark.parametrize("K, N, m", [(320, 160, 1000), (33, 7, 5), (256, 300, 130), (64, 256, 128),
                                     (40, 16, 5), (8, 24, 1), (512, 512, 1024)])
def test_tcgen05_gemm_matches_exact_and_mma_sync(K, N, m):
    """One linear layer (no intermediate rounding): both tcgen05 paths (TMA-fed
    where the widths are multiples of 8, else thread-staged; and the
    thread-staged one forced) equal the float64 product of the same bfloat16
    operands to float32 accumulation error, and agree with the mma.sync path;
    the backward products (transposed operands) likewise. Shapes cover ragged
    M and N, N above one 256-column tile, K below one 64-deep chunk, a
    single row, and widths that are not multiples of 8 (thread staging)."""
    rng = np.random.default_rng(11)
    sizes = [K, N]
    W = rng.standard_normal((K, N)) / np.sqrt(K)
    b = 0.1 * rng.standard_normal(N)
    flat = _flat([(W, b)])
    x = rng.standard_normal((m, K)).astype(np.float32)
    dy = rng.standard_normal((m, N)).astype(np.float32)
    p32 = _unflat(flat, sizes)
    y_ref = om.bf16(x) @ om.bf16(p32[0][0]) + p32[0][1]
    gW_ref = om.bf16(x).T @ om.bf16(dy)
    out = {}
    for tc in (1, 2, 0):
        net = thor.thor_mlp_create(sizes, max(m, 1), seed=0)
        try:
            thor.thor_mlp_tune(net, thor.THOR_MLP_TUNE_TCGEN05, tc)
            thor.thor_mlp_set_params(net, flat)
            yd = torch.empty((m, N), dtype=torch.float32, device="cuda")
            thor.thor_mlp_forward(net, torch.tensor(x, device="cuda"), yd)
            gd = torch.empty(flat.size, dtype=torch.float32, device="cuda")
            thor.thor_mlp_backward(net, torch.tensor(dy, device="cuda"), gd)
            thor.thor_mlp_get_params(net)          # synchronises; raises on a timed-out MMA wait
            out[tc] = (yd.cpu().numpy().astype(np.float64), gd.cpu().numpy().astype(np.float64))
        finally:
            thor.thor_mlp_destroy(net)
    for tc in (1, 2, 0):
        y, g = out[tc]
        assert _rel(y, y_ref) < 1e-5, (tc, _rel(y, y_ref))
        gW = g[:K * N].reshape(K, N)
        assert _rel(gW, gW_ref) < 1e-5, (tc, _rel(gW, gW_ref))
    assert _rel(out[1][0], out[0][0]) < 1e-5
    assert _rel(out[2][0], out[0][0]) < 1e-5
