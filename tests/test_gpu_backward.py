"""GPU tests of the adjoint (htex_lookup_backward) beyond oracle parity:
central finite differences taken with the GPU forward itself, and a texture
fit driven by the gradient."""
import numpy as np
import pytest

import htex_synth as syn
import paper_2207_05618_gb300 as hx

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2207_05618_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def test_backward_matches_gpu_central_differences():
    """L = sum_q g_q . out_q is linear in every texel, so (L(T + e) - L(T - e)) / 2e
    equals dL/dT up to the FP32 rounding of the touched outputs; half the
    checked texels have a nonzero gradient, half are untouched (exactly 0)."""
    fs, fv, V, _ = syn.uv_sphere(slices=12, rings=9, seed=3)
    mesh = hx.Mesh(fs, fv, V)
    log2n = (np.arange(mesh.E) * 7 % 5).astype(np.int32)
    tex_np = syn.texels_f32(log2n, 3, seed=4)
    tex = hx.Textures.upload(mesh, log2n, tex_np, 3, "f32", hx.BUILD_MIPS)
    qs = syn.queries(mesh.H, 40000, seed=5, footprint="loguniform", lo=-5, hi=0.5)
    q = torch.from_numpy(hx.pack_queries(*qs)).cuda()
    g = torch.from_numpy(np.random.default_rng(6).standard_normal((40000, 3)).astype(np.float32)).cuda()
    grad = hx.lookup_backward(tex, q, g).double().cpu().numpy()
    pool = torch.from_numpy(tex.download_pool()[0].view(np.float32).copy()).cuda()
    nz = np.nonzero(grad)[0]
    zero = np.nonzero(grad == 0)[0]
    rng = np.random.default_rng(7)
    picks = np.concatenate([rng.choice(nz, 24, replace=False), rng.choice(zero, 8, replace=False)])
    eps = 1e-2
    gd = g.double()
    for k in picks:
        base = float(pool[k])
        vals = []
        for s in (+1.0, -1.0):
            v = torch.tensor([base + s * eps], dtype=torch.float32, device="cuda")
            tex.write_pool(v, offset=int(k) * 4)
            vals.append((hx.lookup(tex, q).double() * gd).sum().item())
        tex.write_pool(torch.tensor([base], dtype=torch.float32, device="cuda"), offset=int(k) * 4)
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - grad[k]) <= 2e-3 * max(abs(grad[k]), 1.0), (k, fd, grad[k])


def test_write_pool_bounds():
    fs, fv, V, _ = syn.cube()
    mesh = hx.Mesh(fs, fv, V)
    log2n = np.full(mesh.E, 1, np.int32)
    tex = hx.Textures.upload(mesh, log2n, syn.texels_f32(log2n, 1, 1), 1, "f32", hx.BUILD_MIPS)
    with pytest.raises(hx.HtexError):
        tex.write_pool(np.zeros(8, np.uint8), offset=tex.pool_bytes - 4)
    tex.write_pool(np.zeros(4, np.uint8), offset=tex.pool_bytes - 4)


def test_fit_to_smooth_target():
    """Adam on the texels, gradients from the adjoint kernel: lookups of a
    zero-initialised asset approach those of a smooth target asset."""
    from paper_2207_05618_gb300 import fit
    fs, fv, V, _ = syn.uv_sphere(slices=24, rings=16, seed=1)
    mesh = hx.Mesh(fs, fv, V)
    log2n = np.full(mesh.E, 3, np.int32)
    target = hx.Textures.upload(mesh, log2n, syn.texels_smooth(log2n, 3, seed=2), 3, "f32", hx.BUILD_MIPS)
    tex = hx.Textures.upload(mesh, log2n, np.zeros(mesh.E * 64 * 3, np.float32), 3, "f32", hx.BUILD_MIPS)

    def batches(step):
        q = torch.from_numpy(hx.pack_queries(*syn.queries(mesh.H, 200000, seed=100 + step))).cuda()
        return q, hx.lookup(target, q)

    res = fit.fit(tex, batches, steps=80, lr=0.05)
    assert all(np.isfinite(res.losses))
    assert res.ratio < 0.02, res.losses[::10]


def test_sorted_backward_matches_unsorted_and_oracle():
    """HTEX_LOOKUP_BIN on the adjoint: queries sorted by halfedge range in
    chunks of 2^23 with their upstream gradients following them (a full
    chunk plus a ragged one, invalid queries inside), on a pool above the
    64 MiB threshold.  The gradient equals the unsorted kernel's and the
    oracle's up to float-atomic reordering (1e-5 relative to the largest
    entry)."""
    import oracle
    fs, fv, V, _ = syn.cylinder(around=128, rows=60, seed=14)
    mesh = hx.Mesh(fs, fv, V)
    mo = oracle.mesh_from_faces(fs, fv, V)
    log2n = np.full(mesh.E, 5, np.int32)
    tex_np = syn.texels_f32(log2n, 1, seed=15)
    tex = hx.Textures.upload(mesh, log2n, tex_np, 1, "f32", hx.BUILD_MIPS)
    assert tex.pool_bytes > (64 << 20)
    n = (1 << 23) + 4099
    h, u, v, f = syn.queries(mesh.H, n, seed=16, footprint="loguniform", lo=-7, hi=0.5)
    h[::50021] = -1
    q = torch.from_numpy(hx.pack_queries(h, u, v, f)).cuda()
    g = torch.from_numpy(np.random.default_rng(17).standard_normal((n, 1)).astype(np.float32)).cuda()
    s0 = torch.zeros(1, dtype=torch.int32, device="cuda")
    s1 = torch.zeros(1, dtype=torch.int32, device="cuda")
    a = hx.lookup_backward(tex, q, g, status=s0).double().cpu().numpy()
    b = hx.lookup_backward(tex, q, g, flags=hx.LOOKUP_BIN, status=s1).double().cpu().numpy()
    assert int(s0.item()) == int(s1.item()) == int((h < 0).sum())
    scale = np.abs(a).max()
    assert np.abs(a - b).max() <= 1e-5 * scale
    # oracle on the first 200k queries (the gradient is a sum over queries)
    k = 200000
    to = oracle.prepare_textures(mo, log2n, tex_np, 1, "f32", hx.BUILD_MIPS)
    ref = oracle.grad_to_pool_layout(to, oracle.lookup_grad(mo, to, (h[:k], u[:k], v[:k], f[:k]),
                                                            g[:k].cpu().numpy().astype(np.float64)), 4)
    c = hx.lookup_backward(tex, q[:k], g[:k], flags=hx.LOOKUP_BIN).double().cpu().numpy()
    assert np.abs(c - ref[:c.shape[0]]).max() <= 1e-5 * max(np.abs(ref).max(), 1.0)


def test_adam_step_matches_torch_adam():
    """htex_textures_adam_step against torch.optim.Adam (plain PyTorch, the
    same hyper-parameters) over five steps of random gradients: the master
    copy agrees to float rounding, the pool holds the master copy and the
    gradient is cleared after every step."""
    fs, fv, V, _ = syn.uv_sphere(slices=8, rings=6, seed=2)
    mesh = hx.Mesh(fs, fv, V)
    log2n = (np.arange(mesh.E) % 4).astype(np.int32)
    tot = int(sum(4 ** int(k) for k in log2n))
    tex = hx.Textures.upload(mesh, log2n, np.zeros(tot * 3, np.float32), 3, "f32", hx.BUILD_MIPS)
    n = tex.pool_elements
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    start = torch.randn(n, device="cuda", generator=gen)
    ref = start.clone().requires_grad_(True)
    opt = torch.optim.Adam([ref], lr=0.01, betas=(0.8, 0.95), eps=1e-6)
    master, grad = start.clone(), torch.zeros(n, device="cuda")
    m, v = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    for step in range(1, 6):
        g = torch.randn(n, device="cuda", generator=gen) * (10.0 ** (step - 3))
        ref.grad = g.clone()
        opt.step()
        grad.copy_(g)
        tex.adam_step(master, grad, m, v, step, 0.01, betas=(0.8, 0.95), eps=1e-6)
        torch.cuda.synchronize()
        assert torch.count_nonzero(grad) == 0
        assert torch.allclose(master, ref.detach(), rtol=1e-5, atol=1e-6)
        pool = torch.from_numpy(tex.download_pool()[0].view(np.float32).copy()).cuda()
        assert torch.equal(pool, master)
    with pytest.raises(hx.HtexError):
        tex.adam_step(master, grad, m, v, 0, 0.01)
