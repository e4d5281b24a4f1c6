"""GPU checks of the complex gains and the adjoint (differentiable form).

The oracle's FP64 adjoint is itself pinned by central finite differences of
its FP64 forward (tests/oracle_pins.py); here the library's FP32 adjoint is
compared with it, the forward with gains is compared with the oracle's
forward (gains applied to the voltages), and the autograd wrapper is checked
end to end, including a finite-difference check of the GPU forward."""
import numpy as np
import pytest
import torch

import oracle
from paper_1107_4264_gb300 import build as engine_build
from paper_1107_4264_gb300 import synth, xc
from tests.test_parity_gpu import frob_and_maxnorm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    engine_build.build()
    xc.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch.device("cuda:0")


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-30))


@pytest.mark.parametrize("engine", [xc.XC_ENGINE_TENSOR, xc.XC_ENGINE_FP32], ids=["tensor", "fp32"])
def test_forward_with_gains(engine, dev):
    T, F, N, P = 400, 3, 40, 2
    x = synth.sky_voltages(T, F, N, P, noise_sigma=0.7, nsrc=3, src_amp=1.0, seed=61)
    g = synth.complex_gains(N, P, 61)
    want = oracle.correlate_f64(x.double().numpy(), gains=g)
    eng = xc.Correlator(N, P, F, T, "float32", engine=engine)
    try:
        eng.set_gains(torch.from_numpy(g).float().to(dev))
        got = eng.correlate(x.to(dev), sync=True).cpu().double().numpy()
    finally:
        eng.close()
    frob, mx = frob_and_maxnorm(got, want, N, P)
    assert frob <= 1e-3 and mx <= 1e-3, (frob, mx)


def test_gains_rejected_for_8bit_input(dev):
    eng = xc.Correlator(8, 2, 2, 64, "int8")
    try:
        g = torch.ones((8, 2, 2), device=dev)
        with pytest.raises(xc.XcError):
            eng.set_gains(g)
    finally:
        eng.close()


@pytest.mark.parametrize("engine", [xc.XC_ENGINE_TENSOR, xc.XC_ENGINE_FP32], ids=["tensor", "fp32"])
@pytest.mark.parametrize("N,P,F,T", [(12, 2, 3, 70), (7, 1, 2, 33), (70, 2, 2, 130), (130, 2, 2, 300)])
def test_backward_matches_fp64_adjoint(N, P, F, T, engine, dev):
    rng = np.random.default_rng(N * 1000 + T)
    x = rng.standard_normal((T, F, N, P, 2))
    g = synth.complex_gains(N, P, N + T)
    go = rng.standard_normal((F, N * (N + 1) // 2, P * P, 2))
    gx_want, gg_want = oracle.backward_f64(x, go, gains=g)
    eng = xc.Correlator(N, P, F, T, "float32", engine=engine)
    try:
        eng.set_gains(torch.from_numpy(g).float().to(dev))
        gx = eng.correlate_backward(torch.from_numpy(go).float().to(dev),
                                    torch.from_numpy(x).float().to(dev))
        gg = eng.grad_gains()
        torch.cuda.synchronize()
        eng.synchronize()
    finally:
        eng.close()
    assert rel(gx.cpu().double().numpy(), gx_want) <= 2e-5
    assert rel(gg.cpu().double().numpy(), gg_want) <= 2e-5


def _loss(V, M, W):
    d = V - M
    return (W[..., None] * d * d).sum()


def test_autograd_matches_oracle_and_finite_differences(dev):
    """4-station slice: autograd through the FP32 engine against the FP64
    oracle gradient, plus central differences of the GPU forward."""
    T, F, N, P = 64, 2, 4, 2
    rng = np.random.default_rng(7)
    x0 = rng.standard_normal((T, F, N, P, 2))
    g0 = synth.complex_gains(N, P, 7)
    M = rng.standard_normal((F, N * (N + 1) // 2, P * P, 2))
    W = rng.uniform(0, 1, (F, N * (N + 1) // 2, P * P))
    eng = xc.Correlator(N, P, F, T, "float32", engine=xc.XC_ENGINE_FP32)
    try:
        x = torch.from_numpy(x0).float().to(dev).requires_grad_(True)
        g = torch.from_numpy(g0).float().to(dev).requires_grad_(True)
        Mt, Wt = torch.from_numpy(M).float().to(dev), torch.from_numpy(W).float().to(dev)
        L = _loss(xc.correlate_autograd(eng, x, g), Mt, Wt)
        L.backward()
        torch.cuda.synchronize()
        # FP64 reference gradient
        V = oracle.correlate_f64(x0, gains=g0)
        go = 2.0 * W[..., None] * (V - M)
        gx_ref, gg_ref = oracle.backward_f64(x0, go, gains=g0)
        assert rel(x.grad.cpu().double().numpy(), gx_ref) <= 1e-4
        assert rel(g.grad.cpu().double().numpy(), gg_ref) <= 1e-4

        # Central differences of the GPU forward on the linear loss sum W.V:
        # it is quadratic in x and in g, so a central difference is exact
        # for any step and only rounding is left (h = 0.5 keeps it small).
        def lin(xv, gv):
            return (Wt[..., None] * xc.correlate_autograd(eng, xv, gv)).sum()

        xl = x.detach().clone().requires_grad_(True)
        gl = g.detach().clone().requires_grad_(True)
        lin(xl, gl).backward()
        torch.cuda.synchronize()

        def lin_at(xv, gv):
            with torch.no_grad():
                return float(lin(xv, gv).double())

        h = 0.5
        for i in [(3, 1, 2, 1, 0), (10, 0, 0, 0, 1), (40, 1, 3, 1, 1)]:
            xp, xm = x.detach().clone(), x.detach().clone()
            xp[i] += h
            xm[i] -= h
            fd = (lin_at(xp, g.detach()) - lin_at(xm, g.detach())) / (2 * h)
            assert abs(fd - float(xl.grad[i])) <= 1e-2 * max(1.0, abs(fd)), (i, fd, float(xl.grad[i]))
        for i in [(0, 0, 0), (2, 1, 1), (3, 0, 1)]:
            gp, gm = g.detach().clone(), g.detach().clone()
            gp[i] += h
            gm[i] -= h
            fd = (lin_at(x.detach(), gp) - lin_at(x.detach(), gm)) / (2 * h)
            assert abs(fd - float(gl.grad[i])) <= 1e-2 * max(1.0, abs(fd)), (i, fd, float(gl.grad[i]))
    finally:
        eng.close()


def test_differentiable_workload_sampled(dev):
    """Differentiable workload at full size (N=256 x 2 pols, F=64, T=4096):
    loss sum W |V(g x) - M|^2 with M from a second gain set, forward on the
    planar tensor-core engine, backward through the adjoint; grad_x of two
    sampled channels against the FP64 oracle adjoint for the same grad_out."""
    w = synth.DIFF
    x, g, g_t, W = synth.diff_inputs(w, device=dev)
    eng = xc.Correlator(w.nstation, w.npol, w.nfreq, w.ntime, "float32")
    try:
        eng.set_gains(torch.from_numpy(g_t).float().to(dev))
        M = eng.correlate(x, sync=True).clone()
        xg = x.clone().requires_grad_(True)
        gg = torch.from_numpy(g).float().to(dev).requires_grad_(True)
        V = xc.correlate_autograd(eng, xg, gg)
        L = _loss(V, M, W)
        L.backward()
        torch.cuda.synchronize()
        go = (2.0 * W[..., None] * (V.detach() - M)).cpu().double().numpy()
        chans = [5, 41]
        xs = x[:, chans].cpu().double().numpy()
        gx_ref, _ = oracle.backward_f64(xs, go[chans], gains=g)
        got = xg.grad[:, chans].cpu().double().numpy()
        assert rel(got, gx_ref) <= 1e-4
        assert torch.isfinite(gg.grad).all()
    finally:
        eng.close()
