"""Learned warm start on the GPU: gradients against the oracle, training on
the method's own MBFs, and the warm-start gain checked against the FP64 direct MBFs.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle import conv3d  # noqa: E402


def _net(D, H, W, hidden, layers, seed=0, batch=8):
    from paper_2103_08513_gb300.learned import WarmStartNet
    return WarmStartNet(D, H, W, hidden=hidden, layers=layers, batch=batch, seed=seed)


def _oracle_params(net, hidden, layers):
    """The network's parameters as the oracle's layers: BF16 weights (as the
    convolutions use them), FP32 master biases."""
    cin = [4] + [hidden] * (layers - 1)
    cout = [hidden] * (layers - 1) + [1]
    wb = net.bf16_weights().cpu().numpy().astype(np.float64)
    master = net.master.cpu().numpy().astype(np.float64)
    flat = wb.copy()
    off = 0
    for ci, co in zip(cin, cout):
        off += co * ci * 27
        flat[off: off + co] = master[off: off + co]
        off += co
    return conv3d.unflatten(flat, cin, cout)


@pytest.mark.parametrize("shape", [(3, 4, 5, 8, 3, 3), (5, 10, 10, 32, 4, 37)])
def test_gpu_forward_matches_oracle_elementwise(shape):
    """Inference output, element by element, against the oracle's FP64 forward pass
    with the same (BF16-rounded) weights; the GPU accumulates in FP32."""
    D, H, W, hidden, layers, batch = shape
    net = _net(D, H, W, hidden, layers, seed=2, batch=batch)
    rng = np.random.default_rng(7)
    x = torch.from_numpy(rng.normal(size=(batch, 4, D, H, W)).astype(np.float32)).cuda()
    y = net.forward(x)
    torch.cuda.synchronize()
    params = _oracle_params(net, hidden, layers)
    yref = conv3d.forward(params, x.cpu().numpy().astype(np.float64))[-1]
    got = y.cpu().numpy().astype(np.float64).reshape(yref.shape)
    assert np.abs(got - yref).max() <= 2e-6


@pytest.mark.parametrize("weighted", [False, True])
def test_gpu_gradient_matches_oracle(weighted):
    """Loss and gradient against the oracle, without and with the face-flux weights."""
    D, H, W, hidden, layers = 3, 4, 5, 8, 3
    net = _net(D, H, W, hidden, layers)
    rng = np.random.default_rng(1)
    x = torch.from_numpy(rng.normal(size=(3, 4, D, H, W)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.uniform(size=(3, 1, D, H, W)).astype(np.float32)).cuda()
    wn = (rng.uniform(size=(3, 1, D, H, W)) * (rng.uniform(size=(3, 1, D, H, W)) < 0.4)).astype(np.float32)
    wt = torch.from_numpy(wn).cuda() if weighted else None
    grad, loss = net.gradient(x, t, weight=wt)
    torch.cuda.synchronize()
    cin = [4] + [hidden] * (layers - 1)
    cout = [hidden] * (layers - 1) + [1]
    wb = net.bf16_weights().cpu().numpy().astype(np.float64)
    # biases are used in FP32: take them from the master copy
    master = net.master.cpu().numpy().astype(np.float64)
    flat = wb.copy()
    off = 0
    for ci, co in zip(cin, cout):
        off += co * ci * 27
        flat[off: off + co] = master[off: off + co]
        off += co
    params = conv3d.unflatten(flat, cin, cout)
    lref, gref = conv3d.loss_and_grad(params, x.cpu().numpy().astype(np.float64), t.cpu().numpy().astype(np.float64),
                                      wn.astype(np.float64) if weighted else None)
    gref = conv3d.flatten(gref)
    g = grad.cpu().numpy()
    assert abs(float(loss.cpu()[0]) - lref) <= 1e-5 * lref
    assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)


def _mrcm_fields(seeds, n=(40, 40, 10)):
    from synth.fields import lognormal_K
    from synth.wells import corner_wells
    nx, ny, nz = n
    for sd in seeds:
        yield lognormal_K((nz, ny, nx), 2.0, 8.0, 0.1, seed=sd), corner_wells(nx, ny, nz)


def test_training_and_warm_start_gain():
    """Train on the method's own P-MBFs (config-1-style fields), then warm-start CG
    on a held-out field: fewer iterations than from zero, and the CG result agrees
    with the FP64 direct MBFs (the reference) to the CG tolerance."""
    from paper_2103_08513_gb300 import MRCM
    n = (40, 40, 10)
    edges = ([10] * 4, [10] * 4, [5, 5])
    s = MRCM(n, edges, ((5, 2), (5, 2), (5, 2)), precision="fp64")
    net = _net(5, 10, 10, 32, 4, seed=0, batch=256)
    xs, ts = [], []
    for K, f in _mrcm_fields(range(1, 11)):
        s.factor_local(torch.from_numpy(K).cuda())
        s.solve_mbf(torch.from_numpy(f).cuda())
        x, t = net.samples(s)
        xs.append(x.clone()); ts.append(t.clone())
    X = torch.cat(xs)
    T = torch.cat(ts)
    floor = float((T ** 2).mean() - T.mean() ** 2)        # loss of the best constant guess
    net.set_output_bias(float(T.mean()))
    gen = torch.Generator(device="cpu").manual_seed(0)
    for step in range(1000):
        idx = torch.randint(0, X.shape[0], (256,), generator=gen).cuda()
        loss = net.train_step(X[idx].contiguous(), T[idx].contiguous(), lr=1e-3)
    assert float(loss.cpu()[0]) < 0.3 * floor
    # held-out field: CG iterations from the network's guess vs from zero
    K, f = next(_mrcm_fields([201]))
    Kd, fd = torch.from_numpy(K).cuda(), torch.from_numpy(f).cuda()
    s.factor_local(Kd)
    s.solve_mbf(fd)
    x, t = net.samples(s)
    nsm = min(256, x.shape[0])
    y = net.forward(x[:nsm].contiguous())
    it_net = net.pcg(s, y, nsm, maxit=500, tol=1e-6).cpu().numpy()
    _, t_net = net.samples(s)                  # CG results, checked against the direct FP64 MBFs
    s.solve_mbf(fd)
    it_zero = net.pcg(s, None, nsm, maxit=500, tol=1e-6).cpu().numpy()
    assert (it_net <= 500).all() and (it_zero <= 500).all()
    assert it_net.mean() < it_zero.mean()
    err = (t_net[:nsm] - t[:nsm]).norm() / t[:nsm].norm()
    assert float(err) < 1e-4


def _learned_solver(n, edges, patch, **kw):
    from paper_2103_08513_gb300 import MRCM
    return MRCM(n, edges, patch, precision="learned_pcg", ir_tol=1e-9, **kw)


def _learned_solve(s, K, f, net=None, pred=None, cg_maxit=200, max_outer=8):
    Kd, fd = torch.from_numpy(K).cuda(), torch.from_numpy(f).cuda()
    s.factor_local(Kd)
    if net is not None and pred is None:
        x, _ = net.samples(s, targets=False)
        pred = net.predict(x)
    s.solve_mbf_learned(fd, net=net, pred=pred, cg_maxit=cg_maxit, max_outer=max_outer)
    s.assemble_interface()
    X = s.solve_interface()
    p, u, mres = s.reconstruct(X)
    torch.cuda.synchronize()
    return p.cpu().numpy().ravel(), u.cpu().numpy(), X.cpu().numpy()


def test_learned_form_reaches_the_mixed_bar_against_the_oracle():
    """The learned form (CG inside FP64 refinement, every column) matches the
    oracle at 1e-8 with an untrained network's guesses and from zero."""
    import oracle
    from synth.configs import small
    w = small(n=(20, 20, 10), edges=([10, 10], [10, 10], [5, 5]), patch=((5, 2), (5, 2), (5, 2)), sigma=2.0,
              lam=8.0, kz_ratio=0.1)
    prob = oracle.from_workload(w)
    r = oracle.solve_mrcm(prob)
    net = _net(5, 10, 10, 8, 3, seed=0, batch=64)
    for use_net in (True, False):
        s = _learned_solver(w.n, w.edges, w.patch)
        p, u, X = _learned_solve(s, prob.K, prob.f, net=net if use_net else None)
        code, st = s.read_status()
        fb, lost = s.read_fallback()
        ep, eu = np.linalg.norm(p - r.p) / np.linalg.norm(r.p), np.linalg.norm(u - r.u) / np.linalg.norm(r.u)
        print(f"learned (net={use_net}): p {ep:.2e} u {eu:.2e} CG iterations {s.read_cg_iterations()} "
              f"fallback {fb} status {st}")
        assert st["unconverged"] == 0 and lost == 0
        assert ep < 1e-8 and eu < 1e-8


def test_learned_form_falls_back_to_the_direct_solve():
    """With one CG iteration and no refinement step no column reaches the
    tolerance: every subdomain takes the FP64 direct fallback, and the result
    is the FP64 form's."""
    import oracle
    from synth.configs import small
    from gpu_helpers import run_gpu
    w = small(n=(20, 20, 10), edges=([10, 10], [10, 10], [5, 5]), patch=((5, 2), (5, 2), (5, 2)), sigma=2.0,
              lam=8.0, kz_ratio=0.1)
    prob = oracle.from_workload(w)
    s64, p64, u64, X64, *_ = run_gpu(w, prob.K, prob.f, "fp64")
    s = _learned_solver(w.n, w.edges, w.patch, fallback_cap=w.n_sub)
    p, u, X = _learned_solve(s, prob.K, prob.f, cg_maxit=1, max_outer=0)
    assert s.read_fallback() == (w.n_sub, 0)
    assert np.linalg.norm(p - p64) <= 1e-13 * np.linalg.norm(p64)
