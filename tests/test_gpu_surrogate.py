"""Nonthermal coefficients on the GPU: the quadrature against the oracle, the tensor-core
network against its FP64 reference (forward and gradients), and the trained surrogate against
the quadrature it learned from (per-coefficient error, and its speed-up)."""
import math
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import oracle.mlp as M  # noqa: E402

E, ME, C = M.E, M.ME, M.C
# a training box typical of the torus image: ln(nu/nu_c), theta_B, ln Theta_e, kappa
BOX = [-1.0, 0.1, 0.0, 3.2, 11.0, 1.5707, 4.6, 8.0]


@pytest.fixture(scope="module")
def rt():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2302_02733_gb300 import polrt

    torch.cuda.set_device(0)
    ctx = polrt.rt_create(0, torch.cuda.current_stream().cuda_stream)
    yield polrt, ctx
    polrt.rt_destroy(ctx)


def physical(f, ne=1e5, B=10.0):
    """box features -> (ne, Theta, B, nu, theta, kappa) rows"""
    out = np.zeros((len(f), 6))
    nuB = E * B / (2 * math.pi * ME * C)
    for i, (lx, th, lt, k) in enumerate(f):
        Te = math.exp(lt)
        out[i] = (ne, Te, B, math.exp(lx) * 1.5 * nuB * math.sin(th) * Te * Te, th, k)
    return out


def box_points(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(BOX[:4], BOX[4:], (n, 4))


def test_kappa_quadrature_matches_oracle(rt, ora):
    polrt, ctx = rt
    pts = physical(box_points(60, 1))
    pts[::3, 4] = math.pi - pts[::3, 4]          # theta_B beyond pi/2: circular terms flip
    pts[1::7, 5] = 0.0                           # Maxwell-Juttner rows
    out = np.zeros((len(pts), 8))
    polrt.rt_kappa_coeffs(ctx, pts, out)
    worst = 0.0
    for p, g in zip(pts, out):
        ref = ora.kappa_coeffs(*p)
        rel = np.abs(g - ref) / np.maximum(np.abs(ref), 1e-300)
        worst = max(worst, rel.max())
    print(f"kappa quadrature GPU vs oracle: max rel {worst:.2e}")
    assert worst <= 1e-5


def bf16(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.to(torch.float64).numpy()


def forward_bf16(theta, x):
    """the reference network with the GPU's roundings: BF16 weights and layer inputs, FP64 sums"""
    a = bf16(x)
    for li, (W, b) in enumerate(M.unpack(theta)):
        z = a @ bf16(W).T + bf16(b)
        a = bf16(M.silu(z)) if li < 3 else z
    return a


def init_theta(seed):
    rng = np.random.default_rng(seed)
    parts = []
    for o, i in M.SHAPES:
        lim = math.sqrt(3.0 / i)
        parts.append(np.concatenate([rng.uniform(-lim, lim, (o, i)), np.zeros((o, 1))], axis=1).ravel())
    return np.concatenate(parts).astype(np.float32)


def test_tensor_core_forward_matches_reference(rt):
    polrt, ctx = rt
    theta = init_theta(5)
    polrt.rt_mlp_set_params(ctx, theta, polrt.mlp_norm(BOX[:4], BOX[4:]))
    rng = np.random.default_rng(6)
    x = rng.uniform(-1, 1, (1000, 4)).astype(np.float32)  # a ragged last tile
    y = torch.zeros((1000, 8), dtype=torch.float32, device="cuda")
    polrt.rt_mlp_forward(ctx, torch.from_numpy(x).cuda(), y)
    g = y.cpu().numpy().astype(np.float64)
    exact = M.forward(theta.astype(np.float64), x)
    emul = forward_bf16(theta, x)
    rms = np.sqrt((exact ** 2).mean())
    r_emul, m_emul = np.sqrt(((g - emul) ** 2).mean()) / rms, np.abs(g - emul).max() / rms
    r_exact, m_exact = np.sqrt(((g - exact) ** 2).mean()) / rms, np.abs(g - exact).max() / rms
    print(f"tensor-core forward, error of rms output: vs BF16 emulation rms {r_emul:.2e} max {m_emul:.2e}; "
          f"vs FP64 rms {r_exact:.2e} max {m_exact:.2e}")
    # a wrong operand layout gives errors of order one; BF16 rounding flips give a few 1e-3
    assert r_emul <= 3e-3 and m_emul <= 3e-2 and r_exact <= 1e-2 and m_exact <= 6e-2


def test_tensor_core_gradient_matches_reference(rt):
    """P11: the GPU backward (tensor cores, BF16 operands) against the FP64 backward on the same
    weights, layer by layer, within 1e-2 in norm."""
    polrt, ctx = rt
    theta = init_theta(7)
    polrt.rt_mlp_set_params(ctx, theta, polrt.mlp_norm(BOX[:4], BOX[4:]))
    rng = np.random.default_rng(8)
    x = rng.uniform(-1, 1, (640, 4)).astype(np.float32)
    t = rng.normal(0, 1, (640, 8)).astype(np.float32)
    grad = np.zeros(M.NPARAM, dtype=np.float32)
    loss = polrt.rt_mlp_grad(ctx, torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), grad)
    lref, gref = M.loss_and_grad(theta.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    assert abs(loss / lref - 1) < 1e-2, (loss, lref)
    k = 0
    for o, i in M.SHAPES:
        n = o * (i + 1)
        a, b = grad[k:k + n].astype(np.float64), gref[k:k + n]
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        print(f"layer {o}x{i}: gradient rel err {rel:.2e}")
        assert rel <= 1e-2
        k += n


def test_trained_surrogate_against_quadrature(rt, ora):
    polrt, ctx = rt
    n = 1 << 18
    xs = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ys = torch.empty((n, 8), dtype=torch.float32, device="cuda")
    vs = torch.empty((n,), dtype=torch.int32, device="cuda")
    polrt.rt_surrogate_dataset(ctx, BOX, n, 11, xs, ys, vs)
    valid = vs.bool()
    assert valid.float().mean() > 0.99
    xs, ys = xs[valid].contiguous(), ys[valid].contiguous()
    # the dataset's targets against the oracle's quadrature on a few rows
    xh, yh = xs[:6].cpu().numpy(), ys[:6].cpu().numpy()
    f = np.asarray(BOX[:4]) + (xh + 1) / 2 * (np.asarray(BOX[4:]) - np.asarray(BOX[:4]))
    for fi, yi in zip(f, yh):
        p = physical([fi], ne=1.0, B=1.0)[0]
        yo = M.targets(ora.kappa_coeffs(*p), 1.0, p[1], 1.0, p[3], p[4])
        assert np.abs(yi - yo).max() < 2e-3, (yi, yo)
    tn = torch.empty_like(ys)
    ones = torch.ones(len(xs), dtype=torch.int32, device="cuda")
    norm = polrt.rt_surrogate_fit(ctx, xs, ys, ones, tn, BOX[:4], BOX[4:])
    print("baseline residual std per target:", np.round(np.array(norm.y_std[:]), 4))
    polrt.rt_mlp_set_params(ctx, init_theta(12), norm)
    steps = 20000
    curve = np.zeros(steps, dtype=np.float32)
    t0 = time.perf_counter()
    polrt.rt_mlp_train(ctx, xs, tn, steps, 8192, 2e-3, 13, curve)
    train_s = time.perf_counter() - t0
    print(f"training: {steps} steps in {train_s:.2f} s, loss {curve[:10].mean():.3e} -> {curve[-100:].mean():.3e}")
    assert curve[-100:].mean() < 1e-2 * curve[:10].mean()
    # check on fresh points inside the box
    pts = physical(box_points(4096, 21))
    d_in = torch.from_numpy(pts).cuda()
    q = torch.zeros((len(pts), 8), dtype=torch.float64, device="cuda")
    s = torch.zeros_like(q)
    inside = torch.zeros(len(pts), dtype=torch.uint8, device="cuda")
    polrt.rt_kappa_coeffs(ctx, d_in, q)
    polrt.rt_surrogate_coeffs(ctx, d_in, s, inside)
    assert bool(inside.all())
    rel = (torch.abs(s - q) / torch.abs(q).clamp_min(1e-300)).cpu().numpy()
    names = ["jI", "jQ", "jV", "aI", "aQ", "aV", "rQ", "rV"]
    med, p99 = np.median(rel, axis=0), np.percentile(rel, 99, axis=0)
    print("surrogate vs quadrature, median:", dict(zip(names, np.round(med, 5))))
    print("surrogate vs quadrature, p99:   ", dict(zip(names, np.round(p99, 5))))
    assert med.max() <= 1e-2 and p99.max() <= 5e-2
    # what the network gains: coefficients of 2^20 points, quadrature vs surrogate
    big = torch.from_numpy(physical(box_points(1 << 20, 22))).cuda()
    ob = torch.zeros((1 << 20, 8), dtype=torch.float64, device="cuda")
    times = {}
    for name, fn in (("quadrature", lambda: polrt.rt_kappa_coeffs(ctx, big, ob)),
                     ("surrogate", lambda: polrt.rt_surrogate_coeffs(ctx, big, ob))):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        times[name] = time.perf_counter() - t0
    print(f"2^20 points: quadrature {times['quadrature'] * 1e3:.1f} ms, surrogate {times['surrogate'] * 1e3:.1f} ms, "
          f"speed-up {times['quadrature'] / times['surrogate']:.1f}x")
    assert times["surrogate"] * 5 < times["quadrature"]


def test_training_is_reproducible(rt):
    """The gradient of a batch is summed over its 128-sample tiles in a fixed order (no atomics),
    so two training runs from the same parameters and seed give the same network bit for bit,
    and so does the single gradient call twice."""
    polrt, ctx = rt
    rng = np.random.default_rng(41)
    n = 1 << 14
    x = torch.from_numpy(rng.uniform(-1, 1, (n, 4)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.normal(0, 1, (n, 8)).astype(np.float32)).cuda()
    norm = polrt.mlp_norm(BOX[:4], BOX[4:])
    runs = []
    for _ in range(2):
        polrt.rt_mlp_set_params(ctx, init_theta(42), norm)
        curve = np.zeros(300, dtype=np.float32)
        polrt.rt_mlp_train(ctx, x, t, 300, 2048, 2e-3, 43, curve)
        theta = np.zeros(M.NPARAM, dtype=np.float32)
        polrt.rt_mlp_get_params(ctx, theta)
        runs.append((theta, curve))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    assert not np.array_equal(runs[0][0], init_theta(42).astype(np.float32))
    g1, g2 = np.zeros(M.NPARAM, dtype=np.float32), np.zeros(M.NPARAM, dtype=np.float32)
    l1 = polrt.rt_mlp_grad(ctx, x, t, g1)
    l2 = polrt.rt_mlp_grad(ctx, x, t, g2)
    assert np.array_equal(g1, g2) and l1 == l2
