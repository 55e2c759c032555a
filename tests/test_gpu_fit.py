"""GPU parity of the fitting path: fused loss + adjoint (shm_fit_backward), Adam (shm_adam_step) and
the autograd wrappers, against the FP64 oracle (oracle/fit.py, oracle/adjoint.c)."""
import numpy as np
import pytest
import torch

import oracle as O
import oracle.fit as OF
import shm_inputs as I
from gpu_common import shm, upload_pool

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return shm()


def _targets(G, L, dirs, glyph, seed):
    c = I.sh_coeffs(G, L, seed)
    R, _, n = O.sh_eval(L, c, dirs, glyph=glyph)
    return c, R, n


def test_fit_backward_parity(S):
    G, N, per = 3, 12, 3000
    luts = [O.bake_sh(N, 4, I.sh_coeffs(1, 4, 80 + g)[0] + np.eye(1, 25, 0)[0] * 2.0) for g in range(G)]
    L, stored = upload_pool(S, luts)
    dirs = I.directions(G * per, 81)
    glyph = np.repeat(np.arange(G), per).astype(np.int32)
    _, Rt, nt = _targets(G, 8, dirs, glyph, 82)
    Rt32, nt32 = Rt.astype(np.float32), nt.astype(np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dl = S.like_lut(L, zero=True)
    loss = torch.zeros(1, device="cuda")
    S.fit_backward(L, t(dirs), t(Rt32), t(nt32), dl, w_value=1.0, w_normal=0.5, loss=loss,
                   seg=t(I.query_glyphs_csr(G, per)))
    off, Ns = O.make_pool(luts)[1:]
    lref, dref = OF.loss_and_grad(stored.reshape(-1, 4), off, Ns, dirs, Rt32.astype(np.float64),
                                  nt32.astype(np.float64), 1.0, 0.5, glyph=glyph)
    assert abs(loss.item() - lref) <= 1e-5 * lref
    got = dl.data.view(-1, 4).double().cpu().numpy()
    for ch in range(4):
        assert np.abs(got[:, ch] - dref[:, ch]).max() <= 2e-5 * np.abs(dref[:, ch]).max()


def test_adam_parity(S):
    rng = np.random.default_rng(83)
    n = 100003
    p = rng.normal(size=n).astype(np.float32)
    m = (0.1 * rng.normal(size=n)).astype(np.float32)
    v = np.abs(0.01 * rng.normal(size=n)).astype(np.float32)
    g = rng.normal(size=n).astype(np.float32)
    P, G_, M, V = (torch.from_numpy(x.copy()).cuda() for x in (p, g, m, v))
    S.adam_step(P, G_, M, V, lr=1e-2, step=7, zero_grad=True)
    # the kernel takes float32 hyper-parameters (0.999 and 1e-2 are not float32 numbers): give the
    # oracle the same values
    f = lambda x: float(np.float32(x))
    pr, mr, vr = OF.adam(p.astype(np.float64), g.astype(np.float64), m.astype(np.float64), v.astype(np.float64),
                         7, f(1e-2), beta1=f(0.9), beta2=f(0.999), eps=f(1e-8))
    assert np.abs(P.double().cpu().numpy() - pr).max() <= 1e-6 * max(1.0, np.abs(pr).max())
    assert np.abs(M.double().cpu().numpy() - mr).max() <= 1e-6
    assert np.abs(V.double().cpu().numpy() - vr).max() <= 1e-7
    assert torch.count_nonzero(G_) == 0


def test_autograd_matches_adjoint(S):
    N = 10
    lut = O.bake_sh(N, 4, I.sh_coeffs(1, 4, 84)[0] + np.eye(1, 25, 0)[0] * 2.0)
    L, stored = upload_pool(S, [lut])
    dirs = I.directions(5000, 85)
    table = L.data.clone().requires_grad_(True)
    d = torch.from_numpy(dirs).cuda().requires_grad_(True)
    R, G, Nn = S.query_fn(table, d, L)
    rng = np.random.default_rng(86)
    wR, wG, wN = (torch.from_numpy(rng.normal(size=s).astype(np.float32)).cuda() for s in ((5000,), (5000, 3), (5000, 3)))
    ((R * wR).sum() + (G * wG).sum() + (Nn * wN).sum()).backward()
    dref, ddref = O.query_vjp(stored.reshape(-1, 4), [0], [N], dirs, gR=wR.double().cpu().numpy(),
                              gG=wG.double().cpu().numpy(), gn=wN.double().cpu().numpy())
    got = table.grad.view(-1, 4).double().cpu().numpy()
    for ch in range(4):
        assert np.abs(got[:, ch] - dref[:, ch]).max() <= 2e-5 * np.abs(dref[:, ch]).max()
    assert d.grad is not None and torch.isfinite(d.grad).all()


def test_sh_coefficient_gradient_through_the_bake(S):
    """d/dcoeff of a query loss through the bake = build adjoint of the table adjoint (oracle)."""
    N, L, G = 16, 6, 4
    c = torch.from_numpy(I.sh_coeffs(G, L, 87).astype(np.float32)).cuda().requires_grad_(True)
    basis = S.sh_basis(N, L)
    lut = S.alloc_lut(G, N)
    table = S.sh_bake_fn(c, basis, lut, L)
    dirs = I.directions(G * 2000, 88)
    seg = torch.from_numpy(I.query_glyphs_csr(G, 2000)).cuda()
    R, _, _ = S.query_fn(table, torch.from_numpy(dirs).cuda(), lut, seg=seg)
    R.sum().backward()
    glyph = np.repeat(np.arange(G), 2000).astype(np.int32)
    luts = [O.bake_sh(N, L, c[g].detach().double().cpu().numpy()) for g in range(G)]
    pool, off, Ns = O.make_pool(luts)
    dpool, _ = O.query_vjp(pool, off, Ns, dirs, gR=np.ones(len(dirs)), glyph=glyph, want_ddirs=False)
    T = 6 * (N + 2) ** 2
    for g in range(G):
        ref = O.bake_sh_vjp(N, L, dpool[off[g]:off[g] + T].reshape(6, N + 2, N + 2, 4))
        assert np.abs(c.grad[g].double().cpu().numpy() - ref).max() <= 2e-5 * np.abs(ref).max()


def test_short_fit_reduces_loss(S):
    """1 glyph-field slice: tables initialised to the constant c00 Y00 fitted to direct-SH targets."""
    G, N, L, per = 8, 16, 8, 4096
    coeffs = I.sh_coeffs(G, L, 89).astype(np.float32)
    lut = S.alloc_lut(G, N, zero=True)
    lut.data.view(G, -1, 4)[:, :, 0] = torch.from_numpy(coeffs[:, 0] * 0.28209479177387814).cuda()[:, None]
    m, v = torch.zeros_like(lut.data), torch.zeros_like(lut.data)
    dl = S.like_lut(lut, zero=True)
    seg = torch.from_numpy(I.query_glyphs_csr(G, per)).cuda()
    cdev = torch.from_numpy(coeffs).cuda()
    losses = []
    for step in range(1, 61):
        dirs = torch.from_numpy(I.directions(G * per, 1000 + step)).cuda()
        Rt, _, nt = S.sh_eval(L, cdev, dirs, seg=seg)
        loss = torch.zeros(1, device="cuda")
        S.fit_backward(lut, dirs, Rt, nt, dl, w_value=1.0, w_normal=1.0, loss=loss, seg=seg)
        S.adam_step(lut.data, dl.data, m, v, lr=1e-2, step=step)
        losses.append(loss.item() / (G * per))
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])


def test_adam_vector_and_scalar_paths_agree(S):
    """16-byte aligned arrays take 128-bit accesses (with a scalar tail), offset views the scalar
    path; element results are identical."""
    rng = np.random.default_rng(90)
    n = 4099
    base = [rng.normal(size=n + 1).astype(np.float32) for _ in range(4)]
    base[3] = np.abs(base[3])
    A = [torch.from_numpy(b[:n].copy()).cuda() for b in base]          # aligned
    B = [torch.from_numpy(b.copy()).cuda()[1:] for b in base]          # 4-byte offset views
    for b, a in zip(B, A):
        b.copy_(a)
    S.adam_step(A[0], A[1], A[2], A[3], lr=1e-2, step=3, zero_grad=True)
    S.adam_step(B[0], B[1], B[2], B[3], lr=1e-2, step=3, zero_grad=True)
    for a, b in zip(A, B):
        assert torch.equal(a, b)


def test_deterministic_gradients_through_the_bake(S):
    """query_fn(..., deterministic=True): coefficient gradients bit-identical over two backward
    passes, and equal to the atomic pass within float32 summation-order error; without segments the
    deterministic pass is refused."""
    N, L, G, per = 16, 6, 5, 3000
    basis = S.sh_basis(N, L)
    dirs = torch.from_numpy(I.directions(G * per, 90)).cuda()
    seg = torch.from_numpy(I.query_glyphs_csr(G, per)).cuda()
    grads = []
    for det in (True, True, False):
        c = torch.from_numpy(I.sh_coeffs(G, L, 89).astype(np.float32)).cuda().requires_grad_(True)
        lut = S.alloc_lut(G, N)
        table = S.sh_bake_fn(c, basis, lut, L, deterministic=det)
        R, Gd, Nn = S.query_fn(table, dirs, lut, seg=seg, deterministic=det)
        (R.sum() + 0.5 * Gd.square().sum() + Nn[:, 2].sum()).backward()
        grads.append(c.grad.clone())
    assert torch.equal(grads[0], grads[1])
    assert float((grads[0] - grads[2]).abs().max()) <= 1e-5 * float(grads[2].abs().max())
    lut = S.alloc_lut(G, N)
    table = S.sh_bake_fn(torch.zeros((G, (L + 1) ** 2), device="cuda", requires_grad=True), basis, lut, L)
    with pytest.raises(RuntimeError):
        S.query_fn(table, dirs, lut, glyph=torch.zeros(G * per, dtype=torch.int32, device="cuda"), deterministic=True)
