"""Adam step of the mapping iterations (gs_adam_step) through the C ABI vs the FP64 oracle.

FP32 arithmetic against FP64: the moments agree to a few ulp; the update lr m^ / (sqrt(v^) + eps)
is well conditioned away from v = 0, so parameters agree to rtol 1e-5 of the step plus 1e-6
of the value over a few steps."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2409_18122_gb300 import gs

pytestmark = pytest.mark.gpu


def _tensors(seed, shapes):
    rng = np.random.default_rng(seed)
    return [rng.normal(size=s).astype(np.float32) for s in shapes]


def test_adam_steps_vs_oracle_with_a_skipped_tensor():
    shapes = [(1000, 4), (37, 4), (5, 4)]
    p0 = _tensors(1, shapes)
    params = [torch.from_numpy(p).cuda().requires_grad_(True) for p in p0]
    opt = gs.Adam(params, lr=1e-2)
    ref = [(p.astype(np.float64), np.zeros(p.shape), np.zeros(p.shape)) for p in p0]
    rng = np.random.default_rng(2)
    for t in range(1, 5):
        grads = [rng.normal(size=s).astype(np.float32) * (10.0 ** -t) for s in shapes]
        for p, g in zip(params, grads):
            p.grad = torch.from_numpy(g).cuda()
        params[2].grad = None                      # no gradient: tensor 2 is left alone
        opt.step()
        ref = [O.adam_step(rp, g, rm, rv, t, 1e-2) if i != 2 else (rp, rm, rv)
               for i, ((rp, rm, rv), g) in enumerate(zip(ref, grads))]
    torch.cuda.synchronize()
    assert int(opt.step_count.item()) == 4
    for i, (p, (rp, rm, rv)) in enumerate(zip(params, ref)):
        got = p.detach().cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(got, rp, rtol=1e-6, atol=1e-5 * 1e-2)
        # the moment recurrences cancel where a gradient changes sign: FP32 rounding is a few
        # ulp of the terms (bounded by the largest moment), not of the result
        np.testing.assert_allclose(opt.m[i].cpu().numpy(), rm, rtol=1e-5, atol=1e-6 * np.abs(rm).max())
        np.testing.assert_allclose(opt.v[i].cpu().numpy(), rv, rtol=1e-5, atol=1e-6 * np.abs(rv).max())
    np.testing.assert_array_equal(params[2].detach().cpu().numpy(), p0[2])


def test_adam_step_replayed_from_a_graph_advances_the_step():
    """One captured update replayed three times equals three eager oracle steps (the bias
    corrections follow the device step count)."""
    p0 = _tensors(3, [(256, 4)])[0]
    p = torch.from_numpy(p0).cuda().requires_grad_(True)
    g = torch.from_numpy(_tensors(4, [(256, 4)])[0]).cuda()
    p.grad = g
    opt = gs.Adam([p], lr=5e-3)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        opt.step()
    torch.cuda.synchronize()
    # capturing records the kernels without running them: the three replays are steps 1-3
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    assert int(opt.step_count.item()) == 3
    rp, rm, rv = p0.astype(np.float64), np.zeros(p0.shape), np.zeros(p0.shape)
    gn = g.cpu().numpy()
    for t in (1, 2, 3):
        rp, rm, rv = O.adam_step(rp, gn, rm, rv, t, 5e-3)
    np.testing.assert_allclose(p.detach().cpu().numpy(), rp, rtol=1e-6, atol=1e-7)
