"""Reverse-mode differentiation through the C ABI (adjoint plan directions).

The adjoint transforms F^H x and (1/n) F x are bit-exact against the oracle;
the autograd backward pass equals the explicit adjoint bit for bit; gradients
of the quadratic loss sum |F(x) w|^2 (64 signals of n = 2^16 with Gaussian
parts, complex Gaussian weights) agree with central finite differences of the
per-signal loss and with the gradient of torch's own binary64 FFT on the CPU;
torch.autograd.gradcheck / gradgradcheck pass on small cases.
"""
import numpy as np
import pytest

import oracle
from paper_2603_29129_gb300 import build, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def oz():
    build.build()
    from paper_2603_29129_gb300 import ozfft
    ozfft.load()
    return ozfft


@pytest.mark.parametrize("n", [1000, 1024, 1 << 14])
def test_adjoint_directions_bit_exact(oz, n):
    x = synth.complex_signal("uniform", n, 31, batch=2)
    xt = torch.from_numpy(x).cuda()
    for d in (oz.ADJOINT, oz.INVERSE_ADJOINT):
        plan = oz.Plan(n, 2, d)
        y = plan.execute(xt).cpu().numpy()
        for b in range(2):
            yo, _ = oracle.ozfft(x[b], N=plan.N, direction=d)
            assert np.array_equal(y[b].view(np.uint64), yo.view(np.uint64)), (d, b)


def _weights(n, batch, seed):
    return torch.from_numpy(synth.complex_signal("gaussian", n, seed, batch=batch))


def test_backward_is_the_adjoint_transform(oz):
    from paper_2603_29129_gb300 import autograd as ad
    n, B = 3000, 3
    x = torch.from_numpy(synth.complex_signal("gaussian", n, 41, batch=B)).cuda().requires_grad_()
    g = torch.from_numpy(synth.complex_signal("gaussian", n, 42, batch=B)).cuda()
    for fwd, adj in ((ad.fft, oz.ADJOINT), (ad.ifft, oz.INVERSE_ADJOINT)):
        x.grad = None
        fwd(x).backward(g)
        ref = oz.Plan(n, B, adj).execute(g)
        assert np.array_equal(x.grad.cpu().numpy().view(np.uint64), ref.cpu().numpy().view(np.uint64))
    # the package-level fft routes through the same Function when grad is needed
    x.grad = None
    oz.fft(x).backward(g)
    assert np.array_equal(x.grad.cpu().numpy().view(np.uint64),
                          oz.Plan(n, B, oz.ADJOINT).execute(g).cpu().numpy().view(np.uint64))


def test_gradcheck_small(oz):
    from paper_2603_29129_gb300 import autograd as ad
    for n in (16, 12):
        x = torch.from_numpy(synth.complex_signal("gaussian", n, 51, batch=2)).cuda().requires_grad_()
        assert torch.autograd.gradcheck(ad.fft, (x,), eps=1e-6, atol=1e-8, rtol=1e-7)
        assert torch.autograd.gradcheck(ad.ifft, (x,), eps=1e-6, atol=1e-8, rtol=1e-7)
        assert torch.autograd.gradgradcheck(ad.fft, (x,), eps=1e-6, atol=1e-8, rtol=1e-7)


def test_quadratic_loss_gradient_n65536(oz):
    """Loss sum_k |F(x)_k w_k|^2 over 64 signals of n = 2^16 (Gaussian parts,
    seed 5; complex Gaussian weights, seed 6).  PyTorch's conjugate-Wirtinger
    convention gives grad = 2 F^H(|w|^2 . F x)."""
    from paper_2603_29129_gb300 import autograd as ad
    n, B = 1 << 16, 64
    xh = torch.from_numpy(synth.complex_signal("gaussian", n, 5, batch=B))
    w = _weights(n, B, 6)
    x = xh.cuda().requires_grad_()
    wd = w.cuda()
    loss = (ad.fft(x) * wd).abs().square().sum()
    loss.backward()
    g = x.grad.cpu()
    # torch's binary64 FFT on the CPU, through its own autograd
    xc = xh.clone().requires_grad_()
    (torch.fft.fft(xc) * w).abs().square().sum().backward()
    gc = xc.grad
    assert (torch.linalg.vector_norm(g - gc) / torch.linalg.vector_norm(gc)).item() <= 1e-14
    # the closed form, evaluated with the library's own transforms
    y = oz.fft(xh.cuda())
    gf = 2 * oz.Plan(n, B, oz.ADJOINT).execute(((wd.abs() ** 2) * y).contiguous()).cpu()
    assert (torch.linalg.vector_norm(g - gf) / torch.linalg.vector_norm(gf)).item() <= 1e-15
    # central finite differences (h = 1e-6) of the per-signal loss at 64 sampled real coordinates
    rng = np.random.default_rng(7)
    plan1 = oz.Plan(n, 1, oz.FORWARD)
    rms = torch.sqrt((g.abs() ** 2).mean()).item()
    h = 1e-6
    for _ in range(64):
        b, j, part = int(rng.integers(B)), int(rng.integers(n)), int(rng.integers(2))
        e = torch.zeros(n, dtype=torch.complex128)
        e[j] = h if part == 0 else 1j * h
        lb = []
        for s in (1, -1):
            xp = (xh[b] + s * e).cuda()
            lb.append(((plan1.execute(xp) * wd[b]).abs().square().sum()).item())
        fd = (lb[0] - lb[1]) / (2 * h)
        an = g[b, j].real.item() if part == 0 else g[b, j].imag.item()
        assert abs(fd - an) <= 1e-4 * rms, (b, j, part, fd, an)
