"""GPU parity of the right preconditioners: Jacobi, and the learned convolutional network with
flexible RGMRES (its forward pass, loss gradient and Adam step against ``oracle/convnet.py``)."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import paper_2011_05090_gb300 as rgs
from paper_2011_05090_gb300 import learned
import synth
from oracle import convnet as oc
from oracle import gmres as og
from oracle.sketch import Sketch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_2011_05090_gb300 import build
    build.build()
    return rgs.rgs_create()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def dev(v, dtype=torch.float64):
    return torch.tensor(np.asarray(v), dtype=dtype, device="cuda")


def random_params(seed, bias=0.05):
    p = oc.init_params(seed)
    g = np.random.default_rng(seed + 100)
    o = 0
    for co, ci in oc.layer_shapes():
        o += co * ci * 9
        p[o:o + co] = bias * g.standard_normal(co)
        o += co
    return p.astype(np.float32)


def net_batch(B, H, W, seed):
    g = np.random.default_rng(seed)
    x = g.standard_normal((B, 2, H, W)).astype(np.float32)
    return x


def layer_slices():
    out, o = [], 0
    for co, ci in oc.layer_shapes():
        n = co * ci * 9 + co
        out.append(slice(o, o + n))
        o += n
    return out


# ------------------------------------------------------------------ network
def test_params_roundtrip_and_init(h):
    net = rgs.rgs_convnet_create(h, 16, 32, 1, seed=11)
    p = rgs.rgs_convnet_get_params(h, net)
    assert p.dtype == np.float32 and p.size == oc.num_params() == rgs.rgs_convnet_num_params()
    for (co, ci), sl in zip(oc.layer_shapes(), layer_slices()):
        w, b = p[sl][:co * ci * 9], p[sl][co * ci * 9:]
        bound = 1.0 / np.sqrt(9 * ci)
        assert np.all(b == 0) and np.abs(w).max() <= bound and np.abs(w).max() > 0.9 * bound
        assert abs(w.mean()) <= 4 * bound / np.sqrt(3 * w.size)
    q = random_params(3)
    rgs.rgs_convnet_set_params(h, net, q)
    assert np.array_equal(rgs.rgs_convnet_get_params(h, net), q)
    with pytest.raises(rgs.RgsError):
        rgs.rgs_convnet_create(h, 12, 32, 1)                      # H not a multiple of 8
    with pytest.raises(rgs.RgsError):
        rgs.rgs_convnet_create(h, 16, 40, 1)                      # W not a multiple of 16


@pytest.mark.parametrize("H,W,B", [(8, 16, 1), (16, 32, 2), (24, 48, 3), (40, 16, 1)])
def test_forward_matches_oracle(h, H, W, B):
    net = rgs.rgs_convnet_create(h, H, W, B, seed=1)
    p = random_params(H + W)
    rgs.rgs_convnet_set_params(h, net, p)
    x = net_batch(B, H, W, 7)
    out = rgs.rgs_convnet_forward(h, net, dev(x, torch.float32)).cpu().numpy()
    ref_bf, _, _ = oc.forward(p.astype(np.float64), x, bf16=True)
    ref, _, _ = oc.forward(p.astype(np.float64), x)
    e_bf, e = rel(out, ref_bf), rel(out, ref)
    print(f"H={H} W={W} B={B}: vs bf16-rounded oracle {e_bf:.2e}, vs FP64 oracle {e:.2e}")
    # tensor-core sums differ from exact ones by ~1e-6 relative, which flips a few bf16 roundings
    # of the hidden activations (one flip = 2^-8 relative): ~1e-3 end to end
    assert e_bf <= 6e-3 and e <= 3e-2


@pytest.mark.parametrize("H,W,B", [(24, 48, 3), (64, 128, 2)])
def test_tma_convolution_bit_identical_to_cp_async(h, H, W, B, monkeypatch):
    """The convolutions with TMA-staged halos (the default) and with halos staged by per-thread
    asynchronous copies (RGS_CONV_TMA=0) issue the same MMAs in the same order: the forward output
    and the loss gradient agree bit for bit (H = 24: the second 16-row tile is half outside the
    grid)."""
    net = rgs.rgs_convnet_create(h, H, W, B, seed=1)
    rgs.rgs_convnet_set_params(h, net, random_params(H + 2 * W))
    x = dev(net_batch(B, H, W, 12), torch.float32)
    t = dev(np.random.default_rng(13).standard_normal((B, H, W)), torch.float32)
    out = {}
    try:
        for mode in ("tma", "cp"):
            if mode == "cp":
                monkeypatch.setenv("RGS_CONV_TMA", "0")
            f = rgs.rgs_convnet_forward(h, net, x).clone()
            L, g = rgs.rgs_convnet_loss_grad(h, net, x, t)
            out[mode] = (f, L, g)
    finally:
        monkeypatch.delenv("RGS_CONV_TMA", raising=False)
    assert torch.equal(out["tma"][0], out["cp"][0])
    assert out["tma"][1] == out["cp"][1] and np.array_equal(out["tma"][2], out["cp"][2])


def test_forward_batch_entries_are_independent(h):
    H, W = 16, 32
    net = rgs.rgs_convnet_create(h, H, W, 3, seed=2)
    x = dev(net_batch(3, H, W, 8), torch.float32)
    full = rgs.rgs_convnet_forward(h, net, x)
    one = rgs.rgs_convnet_forward(h, net, x[1:2].contiguous())
    assert torch.equal(full[1], one[0])


def test_loss_grad_matches_oracle(h):
    H, W, B = 16, 32, 2
    net = rgs.rgs_convnet_create(h, H, W, B, seed=1)
    p = random_params(5)
    rgs.rgs_convnet_set_params(h, net, p)
    x = net_batch(B, H, W, 9)
    t = np.random.default_rng(10).standard_normal((B, H, W)).astype(np.float32)
    L, g = rgs.rgs_convnet_loss_grad(h, net, dev(x, torch.float32), dev(t, torch.float32))
    Lb, gb = oc.loss_grad(p.astype(np.float64), x, t, bf16=True)
    L64, g64 = oc.loss_grad(p.astype(np.float64), x, t)
    assert abs(L - Lb) <= 1e-3 * Lb and abs(L - L64) <= 3e-2 * L64
    for l, sl in enumerate(layer_slices()):
        eb, e = rel(g[sl], gb[sl]), rel(g[sl], g64[sl])
        print(f"layer {l + 1}: gradient vs bf16-rounded oracle {eb:.2e}, vs FP64 oracle {e:.2e}")
        # the activation gradients are stored in bf16 (as on the GPU): against unrounded FP64 the
        # first layers' sums, which cancel heavily, keep only ~1e-1 relative accuracy
        assert eb <= 1.5e-2 and e <= 0.2


def test_residual_loss_grad_matches_oracle(h):
    from paper_2011_05090_gb300 import learned
    H, W, B = 16, 32, 2
    net = rgs.rgs_convnet_create(h, H, W, B, seed=1)
    p = random_params(6)
    rgs.rgs_convnet_set_params(h, net, p)
    x = net_batch(B, H, W, 19)
    t = x[:, 0].copy()
    S = []
    for b in range(B):
        csr = synth.convdiff_csr((H, W), np.exp(np.random.default_rng(b).standard_normal((H, W))),
                                 np.array([4.0 * b, -3.0]))
        (rp, ci, va), Cb = rgs.csr_to_device(*csr)
        Sd = learned.stencil_from_csr(h, Cb, H, W) / (H + 1) ** 2
        assert np.allclose(Sd.cpu().numpy().astype(np.float64), oc.stencil_from_csr(csr, H, W) / (H + 1) ** 2,
                           rtol=1e-6)
        S.append(Sd)
    S = torch.stack(S).contiguous()
    L, g = rgs.rgs_convnet_loss_grad(h, net, dev(x, torch.float32), dev(t, torch.float32), stencil=S)
    S64 = S.cpu().numpy().astype(np.float64)
    Lb, gb = oc.loss_grad(p.astype(np.float64), x, t, bf16=True, stencil=S64)
    L64, g64 = oc.loss_grad(p.astype(np.float64), x, t, stencil=S64)
    assert abs(L - Lb) <= 1e-3 * Lb and abs(L - L64) <= 3e-2 * L64
    for l, sl in enumerate(layer_slices()):
        eb, e = rel(g[sl], gb[sl]), rel(g[sl], g64[sl])
        print(f"layer {l + 1}: residual-loss gradient vs bf16-rounded oracle {eb:.2e}, vs FP64 oracle {e:.2e}")
        assert eb <= 1.5e-2 and e <= 0.2


def test_train_step_is_one_adam_step(h):
    H, W, B = 16, 32, 2
    net = rgs.rgs_convnet_create(h, H, W, B, seed=4)
    x = dev(net_batch(B, H, W, 12), torch.float32)
    t = dev(np.random.default_rng(13).standard_normal((B, H, W)), torch.float32)
    p0 = rgs.rgs_convnet_get_params(h, net).astype(np.float64)
    L, g = rgs.rgs_convnet_loss_grad(h, net, x, t)
    L1 = rgs.rgs_convnet_train_step(h, net, x, t, lr=1e-3)
    assert L1 == L                                                  # deterministic forward and loss
    p1 = rgs.rgs_convnet_get_params(h, net).astype(np.float64)
    ref, _, _ = oc.adam_step(p0, g.astype(np.float64), np.zeros_like(p0), np.zeros_like(p0), 1, 1e-3)
    assert np.abs(p1 - ref).max() <= 1e-6


def test_training_reduces_loss(h):
    H, W, B = 16, 32, 4
    net = rgs.rgs_convnet_create(h, H, W, B, seed=5)
    xs = net_batch(B, H, W, 14)
    x = dev(xs, torch.float32)
    t = dev(xs[:, 0] * 0.5, torch.float32)                          # a linear map the net can represent
    losses = [rgs.rgs_convnet_train_step(h, net, x, t, lr=2e-3) for _ in range(150)]
    print(f"loss {losses[0]:.3f} -> {losses[-1]:.3f}")
    assert losses[-1] < 0.3 * losses[0]


# ------------------------------------------------------------------ Jacobi
def heterogeneous_system(N=32, seed=0):
    csr, lk = synth.diffusion_2d(N, 1.5, 4, seed)
    A = sp.csr_matrix((csr[2], csr[1], csr[0]))
    return csr, A, lk


def test_jacobi_one_cycle_matches_oracle(h):
    csr, A, _ = heterogeneous_system(32, 1)
    n, m, k = A.shape[0], 20, 70
    b = synth.rhs(n, 3)
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    dinv = 1.0 / A.diagonal()
    for kind in ("srht", "gaussian"):
        sk = rgs.rgs_sketch_create(h, kind, n, k, 5)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        rgs.rgmres_set_preconditioner(h, "jacobi")
        try:
            rgs.rgmres_solve(h, sk, C, dev(b), x, restart=m, max_cycles=1, qdtype=torch.float64, fixed_steps=True)
        finally:
            rgs.rgmres_set_preconditioner(h, "none")
        ref = og.rgmres(A, b, Sketch(kind, n, k, 5), restart=m, max_cycles=1, fixed_steps=True,
                        precond=lambda v: dinv * v)
        assert rel(x.cpu().numpy(), ref.x) <= 1e-10


@pytest.mark.parametrize("qdtype", [torch.float64, torch.float32])
def test_jacobi_converges_faster_than_none(h, qdtype):
    csr, A, _ = heterogeneous_system(64, 2)
    n = A.shape[0]
    b = synth.rhs(n, 4)
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    sk = rgs.rgs_sketch_create(h, "srht", n, 120, 6)
    steps = {}
    for pc in ("none", "jacobi"):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        rgs.rgmres_set_preconditioner(h, pc)
        try:
            res = rgs.rgmres_solve(h, sk, C, dev(b), x, restart=40, rtol=1e-8, max_cycles=400, qdtype=qdtype)
        finally:
            rgs.rgmres_set_preconditioner(h, "none")
        xs = x.cpu().numpy()
        assert res["converged"] and np.linalg.norm(b - A @ xs) / np.linalg.norm(b) <= 1e-8
        assert res["fallback_cycle"] == -1
        steps[pc] = res["total_steps"]
    print(steps)
    assert steps["jacobi"] < steps["none"]


def test_jacobi_rejects_zero_diagonal(h):
    n = 64
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.roll(np.arange(n, dtype=np.int32), 1)                   # a permutation: zero diagonal
    (r_, c_, v_), C = rgs.csr_to_device(rp, ci, np.ones(n))
    sk = rgs.rgs_sketch_create(h, "gaussian", n, 30, 1)
    rgs.rgmres_set_preconditioner(h, "jacobi")
    try:
        with pytest.raises(rgs.RgsError):
            rgs.rgmres_solve(h, sk, C, dev(np.ones(n)), torch.zeros(n, dtype=torch.float64, device="cuda"),
                             restart=10, max_cycles=2)
    finally:
        rgs.rgmres_set_preconditioner(h, "none")


# ------------------------------------------------------------------ learned preconditioner (flexible RGMRES)
def learned_setup(h, N=32, seed=0, params_seed=21):
    csr, A, lk = heterogeneous_system(N, seed)
    net = rgs.rgs_convnet_create(h, N, N, 1, seed=params_seed)
    p = random_params(params_seed)
    rgs.rgs_convnet_set_params(h, net, p)
    return csr, A, lk, net, p


def test_flexible_first_direction_is_the_network_output(h):
    # one step: x = z_0 y_0 with z_0 = M(r_0), so x is parallel to the network's output
    csr, A, lk, net, p = learned_setup(h, 32, 3)
    n = A.shape[0]
    b = synth.rhs(n, 5)
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    sk = rgs.rgs_sketch_create(h, "srht", n, 40, 2)
    lkd = dev(lk).contiguous()
    for qdtype in (torch.float64, torch.float32):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        rgs.rgmres_set_preconditioner(h, "learned", net, lkd, flexible=True)
        try:
            rgs.rgmres_solve(h, sk, C, dev(b), x, restart=1, max_cycles=1, qdtype=qdtype, fixed_steps=True)
        finally:
            rgs.rgmres_set_preconditioner(h, "none")
        z = oc.precondition(p.astype(np.float64), b, lk, bf16=True)
        xs = x.cpu().numpy()
        c = xs @ z / (z @ z)
        assert rel(xs, c * z) <= 6e-3


def identity_like_params(seed, noise=0.02):
    """A network close to z = r: h_0 = relu(r), h_1 = relu(-r) carried through the centre taps of
    layers 2-5, out = h_0 - h_1, plus small random weights everywhere else (so it is nonlinear)."""
    p = random_params(seed).astype(np.float64) * noise
    layers = oc.unflatten(p)
    W, b = layers[0]
    W[0, 0, 1, 1], W[1, 0, 1, 1] = 1.0, -1.0
    b[:2] = 0.0
    for l in range(1, 5):
        W, b = layers[l]
        W[0, :, 1, 1] = W[1, :, 1, 1] = 0.0
        W[0, 0, 1, 1] = W[1, 1, 1, 1] = 1.0
        b[:2] = 0.0
    W, b = layers[5]
    W[0, :2] = 0.0
    W[0, 0, 1, 1], W[0, 1, 1, 1] = 1.0, -1.0
    return oc.flatten(layers).astype(np.float32)


def test_flexible_cycle_matches_oracle(h):
    csr, A, lk, net, _ = learned_setup(h, 32, 4)
    p = identity_like_params(31)
    rgs.rgs_convnet_set_params(h, net, p)
    n, m, k = A.shape[0], 12, 60
    b = synth.rhs(n, 6)
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    sk = rgs.rgs_sketch_create(h, "srht", n, k, 3)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    rgs.rgmres_set_preconditioner(h, "learned", net, dev(lk).contiguous(), flexible=True)
    try:
        res = rgs.rgmres_solve(h, sk, C, dev(b), x, restart=m, max_cycles=1, qdtype=torch.float64, fixed_steps=True)
    finally:
        rgs.rgmres_set_preconditioner(h, "none")
    pm = p.astype(np.float64)
    ref = og.rgmres(A, b, Sketch("srht", n, k, 3), restart=m, max_cycles=1, fixed_steps=True,
                    precond=lambda v: oc.precondition(pm, v, lk, bf16=True), flexible=True)
    xs = x.cpu().numpy()
    r_or = ref.true_residuals[1] / ref.true_residuals[0]
    print(f"flexible cycle: x vs oracle {rel(xs, ref.x):.2e}; residual {res['history'][1]:.4e} (oracle {r_or:.4e})")
    assert r_or < 0.9                                               # the network is a usable preconditioner
    assert rel(xs, ref.x) <= 1e-2
    assert abs(res["history"][1] - r_or) <= 1e-2 * r_or
    assert abs(res["history"][1] - np.linalg.norm(b - A @ xs) / np.linalg.norm(b)) <= 1e-10


@pytest.mark.parametrize("qdtype", [torch.float32, torch.bfloat16])
def test_flexible_with_untrained_network_converges(h, qdtype):
    csr, A, lk, net, p = learned_setup(h, 32, 5)
    n = A.shape[0]
    b = synth.rhs(n, 7)
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    sk = rgs.rgs_sketch_create(h, "srht", n, 100, 4)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    rgs.rgmres_set_preconditioner(h, "learned", net, dev(lk).contiguous(), flexible=True)
    try:
        res = rgs.rgmres_solve(h, sk, C, dev(b), x, restart=30, rtol=1e-8, max_cycles=400, qdtype=qdtype)
    finally:
        rgs.rgmres_set_preconditioner(h, "none")
    xs = x.cpu().numpy()
    print(res["cycles"], res["total_steps"], res["fallback_cycle"])
    assert res["converged"] and np.linalg.norm(b - A @ xs) / np.linalg.norm(b) <= 1e-8


def test_constant_network_falls_back(h):
    # every z_j is a multiple of the same constant field: after one cycle the true residual
    # stops decreasing, the solver switches the preconditioner off and still converges
    csr, A, lk, net, p = learned_setup(h, 32, 6)
    q = np.zeros(oc.num_params(), dtype=np.float32)
    q[-1] = 1.0
    rgs.rgs_convnet_set_params(h, net, q)
    n = A.shape[0]
    b = synth.rhs(n, 8)
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    sk = rgs.rgs_sketch_create(h, "srht", n, 100, 5)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    rgs.rgmres_set_preconditioner(h, "learned", net, dev(lk).contiguous(), flexible=True)
    try:
        res = rgs.rgmres_solve(h, sk, C, dev(b), x, restart=30, rtol=1e-8, max_cycles=400, qdtype=torch.float32)
    finally:
        rgs.rgmres_set_preconditioner(h, "none")
    xs = x.cpu().numpy()
    assert res["fallback_cycle"] >= 1
    assert res["converged"] and np.linalg.norm(b - A @ xs) / np.linalg.norm(b) <= 1e-8


def test_learned_requires_flexible_and_matching_grid(h):
    csr, A, lk, net, p = learned_setup(h, 32, 7)
    with pytest.raises(rgs.RgsError):
        rgs.rgmres_set_preconditioner(h, "learned", net, dev(lk).contiguous(), flexible=False)
    small = rgs.rgs_convnet_create(h, 16, 16, 1)
    n = A.shape[0]
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    sk = rgs.rgs_sketch_create(h, "srht", n, 40, 1)
    rgs.rgmres_set_preconditioner(h, "learned", small, dev(np.zeros((16, 16))).contiguous(), flexible=True)
    try:
        with pytest.raises(rgs.RgsError):
            rgs.rgmres_solve(h, sk, C, dev(synth.rhs(n, 1)), torch.zeros(n, dtype=torch.float64, device="cuda"),
                             restart=10, max_cycles=1)
    finally:
        rgs.rgmres_set_preconditioner(h, "none")


def test_trained_network_beats_jacobi_and_none(h):
    # the whole learned-preconditioner loop at 32 x 32: residuals harvested from plain RGMRES
    # solves (right-hand sides from white noise to smooth), residual-norm training with the
    # hand-written kernels, then flexible RGMRES on held-out coefficient fields
    from paper_2011_05090_gb300 import learned
    N, n = 32, 1024
    sk = rgs.rgs_sketch_create(h, "gaussian", n, 100, 1)
    nfields, per, cycles = 12, 6, 3
    inputs = torch.zeros(nfields * per * cycles, 2, N, N, device="cuda")
    stencils = torch.zeros(nfields, 5, N, N, device="cuda")
    field_of = torch.zeros(inputs.shape[0], dtype=torch.int64, device="cuda")
    w = 0
    for f in range(nfields):
        csr, lk = synth.diffusion_2d(N, 1.5, 2, 100 + f)
        (rp, ci, va), C = rgs.csr_to_device(*csr)
        stencils[f] = learned.stencil_from_csr(h, C, N, N)
        g = np.random.default_rng(f)
        for j in range(per):
            corr = [0, 1, 2, 4, 8][j % 5]
            b = synth.gaussian_field((N, N), corr, g.integers(1 << 30)).ravel() if corr else g.standard_normal(n)
            got = learned.harvest(h, sk, C, dev(lk), dev(b), inputs, start=w, cycles=cycles, restart=50)
            field_of[w:w + got] = f
            w += got
    assert w >= nfields * per
    net = rgs.rgs_convnet_create(h, N, N, 16, seed=3)
    losses = learned.train(h, net, inputs[:w], 600, stencils, field_of[:w], batch=16, lr=1e-3)
    assert np.mean(losses[-50:]) < 0.6 * np.mean(losses[:10])
    steps = {"none": [], "jacobi": [], "learned": []}
    for f in range(2):
        csr, lk = synth.diffusion_2d(N, 1.5, 2, 9000 + f)
        (rp, ci, va), C = rgs.csr_to_device(*csr)
        A = sp.csr_matrix((csr[2], csr[1], csr[0]))
        b = synth.rhs(n, 40 + f)
        for pc in steps:
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            res = learned.solve(h, sk, C, dev(b), x, restart=50, rtol=1e-8, max_cycles=200, precond=pc, net=net,
                                logkappa=dev(lk))
            xs = x.cpu().numpy()
            assert res["converged"] and np.linalg.norm(b - A @ xs) / np.linalg.norm(b) <= 1e-8
            steps[pc].append(res["total_steps"])
    print(steps)
    assert sum(steps["learned"]) < sum(steps["jacobi"]) < sum(steps["none"])


def test_stencil_input_and_residual_entry_points_match_the_oracle(h):
    """rgs_csr_to_stencil against the oracle's loop over the rows (and its rejections),
    rgs_convnet_input against r / rms(r) in FP64, rgs_csr_residual against b - A x on the CPU."""
    H, W = 8, 16
    csr = synth.convdiff_csr((H, W), np.exp(np.random.default_rng(14).standard_normal((H, W))), np.array([2.0, -1.0]))
    arrays, C = rgs.csr_to_device(*csr)
    S = learned.stencil_from_csr(h, C, H, W)
    assert np.allclose(S.cpu().numpy().astype(np.float64), oc.stencil_from_csr(csr, H, W), rtol=1e-6, atol=0)
    with pytest.raises(rgs.RgsError):
        learned.stencil_from_csr(h, C, W, H)            # same n, transposed grid: other neighbour offsets
    with pytest.raises(rgs.RgsError):
        learned.stencil_from_csr(h, C, H, 2 * W)        # wrong number of points
    n = H * W
    g = np.random.default_rng(3)
    r, lk = g.standard_normal(n) * 7.5, g.standard_normal(n)
    out = rgs.rgs_convnet_input(h, dev(r), dev(lk)).cpu().numpy().astype(np.float64)
    rms = np.linalg.norm(r) / np.sqrt(n)
    assert np.allclose(out[0], r / rms, rtol=1e-6, atol=1e-7) and np.allclose(out[1], lk, rtol=1e-6, atol=1e-7)
    A = sp.csr_matrix((csr[2], csr[1], csr[0]))
    x, b = g.standard_normal(n), g.standard_normal(n)
    res, nrm = rgs.rgs_csr_residual(h, C, dev(x), dev(b))
    want = b - A @ x
    assert np.allclose(res.cpu().numpy(), want, rtol=1e-13, atol=1e-13 * np.abs(want).max())
    assert abs(nrm - np.linalg.norm(want)) <= 1e-12 * np.linalg.norm(want)
