"""Unrolled FISTA network: forward and backward kernels against the FP64 oracle, the
plain-FISTA special case, training gain, and the KKT-checked fallback."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import rel_err

pytestmark = pytest.mark.gpu


def _problem(seed, M1=8, M2=8, N=20, L1=32, L2=32, count=3, K=8):
    mask = synth.make_mask(np.random.Generator(np.random.PCG64(seed)), M1, M2, N)
    snaps = [synth.make_snapshot(seed * 100 + i, M1, M2, N, L1, L2, 3, 15.0, mask=mask) for i in range(count)]
    return mask, snaps


def _net(lib, mask, snaps, lam_frac=0.1):
    import torch

    from paper_2509_13592_gb300 import learned

    s0 = snaps[0]
    net = learned.UnrolledNet(s0.M1, s0.M2, mask, s0.L1, s0.L2, len(snaps), lam_frac)
    y = torch.from_numpy(np.concatenate([s.y for s in snaps]).astype(np.complex64)).cuda()
    return net, y


def _oracle_params(s, a, t, lam_frac=0.1):
    A = oracle.dictionary(s.mask, s.M1, s.M2, s.L1, s.L2)
    mu = oracle.step_size(A)
    lam = lam_frac * oracle.lambda_max(A, s.y)
    return A, mu * np.asarray(a, float), mu * lam * np.asarray(t, float), mu, lam


def test_unrolled_forward_matches_oracle(lib):
    import torch

    from paper_2509_13592_gb300 import learned

    mask, snaps = _problem(3)
    K = 8
    rng = np.random.default_rng(0)
    a = (0.7 + 0.5 * rng.random(K)).astype(np.float32)
    t = (0.5 + rng.random(K)).astype(np.float32)
    net, y = _net(lib, mask, snaps)
    c = learned.net_forward(net, y, torch.from_numpy(a).cuda(), torch.from_numpy(t).cuda())
    torch.cuda.synchronize()
    out = c.cpu().numpy().reshape(len(snaps), -1)
    for i, s in enumerate(snaps):
        A, mus, ths, _, _ = _oracle_params(s, a, t)
        ref = oracle.unrolled_forward(A, s.y, mus, ths)
        assert rel_err(out[i], ref) <= 1e-4, (i, rel_err(out[i], ref))
    net.close()


def test_unit_multipliers_are_plain_fista(lib):
    """a = t = 1 runs exactly FISTA's K iterations (same kernel, same arithmetic)."""
    import torch

    from paper_2509_13592_gb300 import learned

    mask, snaps = _problem(4, count=2)
    K = 12
    net, y = _net(lib, mask, snaps)
    ones = torch.ones(K, device="cuda")
    c = learned.net_forward(net, y, ones, ones)
    plain = torch.empty_like(c)
    net.solver.solve(y, K, plain, check=False)
    torch.cuda.synchronize()
    assert torch.equal(c, plain)
    net.close()


def test_unrolled_backward_matches_oracle(lib):
    """dLoss/da_k and dLoss/dt_k from the adjoint kernel equal mu dLoss/dmu_k and mu lam dLoss/dtheta_k of
    the oracle's analytic backward (itself pinned by finite differences), summed over the batch."""
    import torch

    from paper_2509_13592_gb300 import learned

    mask, snaps = _problem(5, count=3)
    K = 8
    rng = np.random.default_rng(1)
    a = (0.8 + 0.4 * rng.random(K)).astype(np.float32)
    t = (0.6 + 0.8 * rng.random(K)).astype(np.float32)
    targets = []
    for s in snaps:
        A, _, _, _, lam = _oracle_params(s, np.ones(1), np.ones(1))
        targets.append(oracle.fista(A, s.y, lam, 200))
    net, y = _net(lib, mask, snaps)
    a_t = torch.from_numpy(a).cuda().requires_grad_(True)
    t_t = torch.from_numpy(t).cuda().requires_grad_(True)
    c = learned.net_forward(net, y, a_t, t_t)
    tgt = torch.from_numpy(np.concatenate(targets).astype(np.complex64)).cuda()
    loss = ((c - tgt).abs() ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    ga = np.zeros(K)
    gt = np.zeros(K)
    for i, s in enumerate(snaps):
        A, mus, ths, mu, lam = _oracle_params(s, a, t)
        ci = oracle.unrolled_forward(A, s.y, mus, ths)
        d_mu, d_th = oracle.unrolled_backward(A, s.y, mus, ths, 2.0 * (ci - targets[i]))
        ga += mu * d_mu
        gt += mu * lam * d_th
    got_a = a_t.grad.cpu().numpy()
    got_t = t_t.grad.cpu().numpy()
    scale = max(np.abs(ga).max(), np.abs(gt).max())
    assert np.abs(got_a - ga).max() <= 2e-3 * scale, (got_a, ga)
    assert np.abs(got_t - gt).max() <= 2e-3 * scale, (got_t, gt)
    net.close()


def test_training_gain_and_kkt_fallback(lib, tmp_path):
    """A short training run on a 64x64 grid makes the 8-layer network closer to 300-iteration FISTA than
    plain FISTA with twice as many (16) iterations, on held-out snapshots; resuming from the checkpoint
    continues; and the KKT-checked fallback refines every snapshot whose residual is above the tolerance."""
    import torch

    from paper_2509_13592_gb300 import learned

    cfg = learned.TrainConfig(M1=16, M2=16, N=64, L1=64, L2=64, layers=8, batch=32, steps=55, target_iters=300,
                              lam_frac=0.1, lr=0.05, checkpoint=str(tmp_path / "ck.pt"), checkpoint_every=10)
    a, t, hist = learned.train(cfg, log=None)
    assert hist[-1] < hist[0]
    cfg2 = learned.TrainConfig(**{**cfg.__dict__, "steps": 60})
    a2, t2, hist2 = learned.train(cfg2, resume=True, log=None)
    assert len(hist2) == 5
    mask = learned.fixed_mask(cfg)
    nb = 64
    y = learned.snapshot_batch(cfg, mask, 10**6, nb)
    ref = learned.plain_fista(cfg, mask, y, 300, nb)
    plain16 = learned.plain_fista(cfg, mask, y, 16, nb)
    net = learned.UnrolledNet(cfg.M1, cfg.M2, mask, cfg.L1, cfg.L2, nb, cfg.lam_frac)
    with torch.no_grad():
        out = learned.net_forward(net, y, a2, t2)
    e_net = learned.relative_errors(out, ref, nb, net.L).mean().item()
    e_plain = learned.relative_errors(plain16, ref, nb, net.L).mean().item()
    assert e_net < e_plain, (e_net, e_plain)
    c, kkt, fell_back = learned.infer_with_fallback(net, y, a2, t2, kkt_tol=0.05, fallback_iters=500)
    assert np.array_equal(fell_back, kkt > 0.05)
    # the fallback answers are FISTA warm-started from the network: closer to the reference than the
    # network's own output for those snapshots
    if fell_back.any():
        idx = torch.as_tensor(np.flatnonzero(fell_back), device="cuda")
        e_after = learned.relative_errors(c.reshape(nb, -1)[idx].reshape(-1), ref.reshape(nb, -1)[idx].reshape(-1),
                                          len(idx), net.L)
        e_before = learned.relative_errors(out.reshape(nb, -1)[idx].reshape(-1),
                                           ref.reshape(nb, -1)[idx].reshape(-1), len(idx), net.L)
        assert e_after.mean() < e_before.mean()
    net.close()


def test_unrolled_grad_y_matches_finite_differences(lib):
    """dLoss/dy through the network (bccb_unrolled_bwd's grad_y) against central differences of
    the FP64 oracle's forward pass in which, as on the GPU, lam = 0.1 ||A^H y||_inf and with it
    every threshold follows the perturbed measurements."""
    import torch

    from paper_2509_13592_gb300 import learned

    mask, snaps = _problem(6, count=2)
    K = 6
    rng = np.random.default_rng(2)
    a = (0.8 + 0.4 * rng.random(K)).astype(np.float32)
    t = (0.6 + 0.8 * rng.random(K)).astype(np.float32)
    targets = []
    for s in snaps:
        A, _, _, _, lam = _oracle_params(s, np.ones(1), np.ones(1))
        targets.append(oracle.fista(A, s.y, lam, 200))
    net, y = _net(lib, mask, snaps)
    y_t = y.clone().requires_grad_(True)
    c = learned.net_forward(net, y_t, torch.from_numpy(a).cuda(), torch.from_numpy(t).cuda())
    tgt = torch.from_numpy(np.concatenate(targets).astype(np.complex64)).cuda()
    ((c - tgt).abs() ** 2).sum().backward()
    torch.cuda.synchronize()
    got = y_t.grad.cpu().numpy().reshape(len(snaps), -1)
    for i, s in enumerate(snaps):
        A = oracle.dictionary(s.mask, s.M1, s.M2, s.L1, s.L2)
        mu = oracle.step_size(A)
        y0 = s.y.astype(np.complex64).astype(np.complex128)  # the measurements the GPU was given

        def loss(yy):
            lam = 0.1 * oracle.lambda_max(A, yy)
            ci = oracle.unrolled_forward(A, yy, mu * a.astype(float), mu * lam * t.astype(float))
            return float(np.sum(np.abs(ci - targets[i]) ** 2))

        h = 1e-6 * np.abs(y0).max()
        fd = np.zeros(y0.size, np.complex128)
        for n in range(y0.size):
            for unit in (1.0, 1j):
                e = np.zeros(y0.size, np.complex128)
                e[n] = h * unit
                d = (loss(y0 + e) - loss(y0 - e)) / (2 * h)
                fd[n] += d * (1.0 if unit == 1.0 else 1j)
        scale = np.abs(fd).max()
        assert scale > 0
        assert np.abs(got[i] - fd).max() <= 2e-3 * scale, (i, np.abs(got[i] - fd).max() / scale)
    net.close()
