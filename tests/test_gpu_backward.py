"""GPU tests of the adjoint (htex_lookup_backward): the FP64 oracle's
gradient, central finite differences taken with the GPU forward itself
(small mesh and the differentiation workload of 2M queries on the ~104k
halfedge sphere), the sorted warp-aggregated path against the plain one,
the torch.autograd.Function, and a texture fit driven by the gradient."""
import numpy as np
import pytest

import htex_synth as syn
import oracle
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
    chunks of 2^24 with their upstream gradients following them (a full
    chunk plus a ragged one, invalid queries inside), on a pool above the
    64 MiB threshold.  The gradient equals the unsorted kernel's and the
    oracle's up to float-atomic reordering (1e-5 relative to the largest
    entry)."""
    fs, fv, V, _ = syn.cylinder(around=128, rows=60, seed=14)
    mesh = hx.Mesh(fs, fv, V)
    mo = oracle.mesh_from_faces(fs, fv, V)
    log2n = np.full(mesh.E, 5, np.int32)
    tex_np = syn.texels_f32(log2n, 1, seed=15)
    tex = hx.Textures.upload(mesh, log2n, tex_np, 1, "f32", hx.BUILD_MIPS)
    assert tex.pool_bytes > (64 << 20)
    n = (1 << 24) + 4099
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


@pytest.mark.parametrize("C,offsets", [(3, (0, 1, 2)), (2, (0, 2)), (1, (0, 1)), (4, (0,))])
def test_backward_every_gradient_alignment(C, offsets):
    """The adjoint into gradient buffers starting 16-, 8- and 4-byte aligned
    (the widest atomics each allows: a float4 for a three-channel texel or a
    pair of two-channel texels when 16-byte aligned, float2 pairs when
    8-byte aligned, scalars otherwise), plain and sorted, on every
    resolution 1..16 with trilinear footprints: each equals the FP64
    oracle's gradient (1e-5 of its largest entry), and the elements before
    and after the buffer stay untouched."""
    gen = lambda: syn.uv_sphere(slices=12, rings=9, seed=3)
    fs, fv, V, _ = gen()
    mesh = hx.Mesh(fs, fv, V)
    mo = oracle.mesh_from_faces(fs, fv, V)
    log2n = (np.arange(mesh.E) * 7 % 5).astype(np.int32)
    tex_np = syn.texels_f32(log2n, C, seed=40 + C)
    tex = hx.Textures.upload(mesh, log2n, tex_np, C, "f32", hx.BUILD_MIPS)
    to = oracle.prepare_textures(mo, log2n, tex_np, C, "f32", hx.BUILD_MIPS)
    n = 30000
    qs = syn.queries(mesh.H, n, seed=41, footprint="loguniform", lo=-5, hi=0.5)
    g = np.random.default_rng(42).standard_normal((n, C)).astype(np.float32)
    ref = oracle.grad_to_pool_layout(to, oracle.lookup_grad(mo, to, qs, g.astype(np.float64)), 4)
    q = torch.from_numpy(hx.pack_queries(*qs)).cuda()
    gd = torch.from_numpy(g).cuda()
    m = tex.pool_elements
    for off in offsets:
        for flags in (0, hx.LOOKUP_BIN):
            base = torch.full((m + 8,), 7.0, dtype=torch.float32, device="cuda")
            grad = base[off:off + m]
            grad.zero_()
            assert grad.data_ptr() % 16 == 4 * off
            hx.lookup_backward(tex, q, gd, grad_texels=grad, flags=flags)
            torch.cuda.synchronize()
            got = grad.double().cpu().numpy()
            assert np.abs(got - ref).max() <= 1e-5 * max(np.abs(ref).max(), 1.0), (off, flags)
            rest = torch.cat([base[:off], base[off + m:]]).cpu().numpy()
            assert np.all(rest == 7.0), (off, flags)
    tex.close()


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


def test_adam_step_in_place_on_the_pool():
    """htex_textures_adam_step with no separate copy (master NULL): the
    pool's own values follow torch.optim.Adam exactly as the master copy
    does in the test above, and the gradient is cleared."""
    fs, fv, V, _ = syn.uv_sphere(slices=8, rings=6, seed=2)
    mesh = hx.Mesh(fs, fv, V)
    log2n = (np.arange(mesh.E) % 4).astype(np.int32)
    tot = int(sum(4 ** int(k) for k in log2n))
    tex = hx.Textures.upload(mesh, log2n, np.zeros(tot * 3, np.float32), 3, "f32", hx.BUILD_MIPS)
    n = tex.pool_elements
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    start = torch.randn(n, device="cuda", generator=gen)
    tex.write_pool(start)
    ref = start.clone().requires_grad_(True)
    opt = torch.optim.Adam([ref], lr=0.02, betas=(0.9, 0.99), eps=1e-7)
    grad = torch.zeros(n, device="cuda")
    m, v = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    for step in range(1, 6):
        g = torch.randn(n, device="cuda", generator=gen)
        ref.grad = g.clone()
        opt.step()
        grad.copy_(g)
        tex.adam_step(None, grad, m, v, step, 0.02, betas=(0.9, 0.99), eps=1e-7)
        torch.cuda.synchronize()
        assert torch.count_nonzero(grad) == 0
        pool = torch.from_numpy(tex.download_pool()[0].view(np.float32).copy()).cuda()
        assert torch.allclose(pool, ref.detach(), rtol=1e-5, atol=1e-6)


U32 = 2.0 ** -24   # unit roundoff of float32


def _pool_index(to):
    """For every pool element (float32 pool of an FP32 asset), the index of
    the same texel value in the oracle's layout, -1 for padding."""
    idx = oracle.grad_to_pool_layout(to, np.arange(1, to.values.size + 1, dtype=np.float64), 4)
    return idx.astype(np.int64) - 1


def test_autograd_function_matches_oracle():
    """HtexLookup through torch.autograd: the forward writes the given
    texel tensor into the resident pool, so its result is the oracle's
    lookup of exactly those values (every level given, no mips built), and
    loss.backward() leaves the oracle's gradient in texels.grad.  Two rounds
    with different texel values show that nothing stale is read."""
    fs, fv, V, _ = syn.uv_sphere(slices=12, rings=9, seed=3)
    mesh = hx.Mesh(fs, fv, V)
    mo = oracle.mesh_from_faces(fs, fv, V)
    log2n = (np.arange(mesh.E) * 7 % 5).astype(np.int32)
    tex = hx.Textures.upload(mesh, log2n, syn.texels_f32(log2n, 3, seed=4), 3, "f32", hx.BUILD_MIPS)
    n = 30000
    qs = syn.queries(mesh.H, n, seed=5, footprint="loguniform", lo=-5, hi=0.5)
    q = torch.from_numpy(hx.pack_queries(*qs)).cuda()
    g = np.random.default_rng(6).standard_normal((n, 3)).astype(np.float32)
    gt = torch.from_numpy(g).cuda()
    layout = oracle.prepare_textures(mo, log2n, np.zeros(int(oracle.texture_offsets(log2n)[-1]) * 3, np.float32),
                                     3, "f32", 0, levels_given=True)
    pidx = _pool_index(layout)
    real = pidx >= 0
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    for scale, offset in ((1.0, 0.0), (2.0, 1.0)):
        texels = (torch.rand(tex.pool_elements, device="cuda", generator=gen) * scale + offset).requires_grad_(True)
        out = hx.HtexLookup.apply(texels, tex, q, 0)
        (out * gt).sum().backward()
        vals = np.zeros(layout.values.size, np.float32)
        vals[pidx[real]] = texels.detach().cpu().numpy()[real]
        to = oracle.prepare_textures(mo, log2n, vals, 3, "f32", 0, levels_given=True)
        ref = oracle.lookup(mo, to, qs)
        assert np.abs(out.detach().cpu().numpy() - ref).max() <= 1e-5 * max(1.0, scale + offset)
        gref = oracle.grad_to_pool_layout(to, oracle.lookup_grad(mo, to, qs, g.astype(np.float64)), 4)
        got = texels.grad.double().cpu().numpy()
        assert np.abs(got - gref).max() <= 1e-5 * np.abs(gref).max()
        assert np.all(got[~real] == 0)
    with pytest.raises(ValueError):
        hx.HtexLookup.apply(torch.zeros(7, device="cuda"), tex, q, 0)


def test_differentiation_workload_oracle_gradient_and_central_differences():
    """The differentiation workload as specified: the closed UV sphere
    (160 x 160 with splits and merges, about 104k halfedges), 32x32 RGB FP32
    textures, 2M level-0 queries, upstream gradient N(0, 1).

    1. The sorted, warp-aggregated adjoint (HTEX_LOOKUP_BIN) equals the
       FP64 oracle's gradient over all 2M queries to 1e-5 of the largest
       entry (float atomics reorder the sums).
    2. Central differences of the GPU forward, eps = 1e-3, on 512 texels:
       256 drawn from texels with a nonzero oracle gradient and 256 from
       texels no query touches.  L = sum g . out is linear in each texel, so
       (L(T + eps) - L(T - eps)) / (T+ - T-) is its derivative up to the
       float32 rounding of the two forward passes; the difference of the
       two passes is taken per output in FP64 on the GPU.  Only the outputs
       after the perturbed tap differ between the passes: at most m = 16
       taps of fused multiply-adds and one product with the common 1/W, so
       |out+ - out-  - exact| <= (2m + 2) u max|T| per output, and
       |fd - dL/dT| <= (2m + 2) u max|T| sum|g| / (T+ - T-) over the outputs
       that changed.  Untouched texels: both the differences and the
       gradient are exactly 0."""
    fs, fv, V, _ = syn.uv_sphere()
    mesh = hx.Mesh(fs, fv, V)
    assert 100_000 <= mesh.H <= 110_000
    mo = oracle.mesh_from_faces(fs, fv, V)
    log2n = np.full(mesh.E, 5, np.int32)
    tex_np = syn.texels_f32(log2n, 3, seed=41)
    tex = hx.Textures.upload(mesh, log2n, tex_np, 3, "f32", hx.BUILD_MIPS)
    n = 2_000_000
    h, u, v, f = syn.queries(mesh.H, n, seed=42)
    q = torch.from_numpy(hx.pack_queries(h, u, v, f)).cuda()
    g = np.random.default_rng(43).standard_normal((n, 3)).astype(np.float32)
    gt = torch.from_numpy(g).cuda()
    grad = hx.lookup_backward(tex, q, gt, flags=hx.LOOKUP_BIN).double().cpu().numpy()
    to = oracle.prepare_textures(mo, log2n, tex_np, 3, "f32", hx.BUILD_MIPS)
    ref = oracle.grad_to_pool_layout(to, oracle.lookup_grad(mo, to, (h, u, v, f), g.astype(np.float64)), 4)
    scale = np.abs(ref).max()
    assert np.abs(grad - ref).max() <= 1e-5 * scale

    real = _pool_index(to) >= 0
    rng = np.random.default_rng(44)
    picks = np.concatenate([rng.choice(np.flatnonzero(ref != 0), 256, replace=False),
                            rng.choice(np.flatnonzero((ref == 0) & real), 256, replace=False)])
    pool = tex.download_pool()[0].view(np.float32).copy()
    maxT = float(np.abs(pool).max()) + 1e-3
    gd = gt.double()
    gabs = gd.abs().sum(1)
    eps = 1e-3
    worst = 0.0
    for k in picks:
        base = np.float32(pool[k])
        tp, tm = np.float32(base + np.float32(eps)), np.float32(base - np.float32(eps))
        outs = []
        for val in (tp, tm):
            tex.write_pool(np.array([val], np.float32), offset=int(k) * 4)
            outs.append(hx.lookup(tex, q).double())
        tex.write_pool(np.array([base], np.float32), offset=int(k) * 4)
        d = outs[0] - outs[1]
        delta = float(tp) - float(tm)
        fd = float((d * gd).sum()) / delta
        if ref[k] == 0:
            assert fd == 0.0 and grad[k] == 0.0, (k, fd, grad[k])
            continue
        changed = (d != 0).any(1)
        bound = 34 * U32 * maxT * float(gabs[changed].sum()) / delta + 1e-5 * scale
        err = abs(fd - grad[k])
        worst = max(worst, err / bound)
        assert err <= bound, (k, fd, grad[k], bound)
    print(f"central differences: largest error {worst:.3g} of its bound")


@pytest.mark.parametrize("channels", [3, 4])
def test_sorted_aggregated_backward_on_shared_levels(channels):
    """Many queries per texture with footprints reaching the coarse levels:
    after the sort by texture, most lanes of a warp share their coarse-level
    taps, so the warp-aggregated atomics merge them.  The gradient equals
    the plain per-lane adjoint's and the oracle's (1e-5 of the largest
    entry); invalid queries are counted once each."""
    fs, fv, V, _ = syn.cylinder(around=24, rows=6, seed=8)
    mesh = hx.Mesh(fs, fv, V)
    mo = oracle.mesh_from_faces(fs, fv, V)
    log2n = np.full(mesh.E, 7, np.int32)
    tex_np = syn.texels_f32(log2n, channels, seed=9)
    tex = hx.Textures.upload(mesh, log2n, tex_np, channels, "f32", hx.BUILD_MIPS | hx.MIRROR_BOUNDARY)
    assert tex.pool_bytes > (64 << 20)
    n = (1 << 21) + 999
    h, u, v, f = syn.queries(mesh.H, n, seed=10, footprint="loguniform", lo=-9, hi=0.5)
    h[::7919] = -1
    q = torch.from_numpy(hx.pack_queries(h, u, v, f)).cuda()
    g = np.random.default_rng(11).standard_normal((n, channels)).astype(np.float32)
    gt = torch.from_numpy(g).cuda()
    s0 = torch.zeros(1, dtype=torch.int32, device="cuda")
    s1 = torch.zeros(1, dtype=torch.int32, device="cuda")
    a = hx.lookup_backward(tex, q, gt, status=s0).double().cpu().numpy()
    b = hx.lookup_backward(tex, q, gt, flags=hx.LOOKUP_BIN, status=s1).double().cpu().numpy()
    assert int(s0.item()) == int(s1.item()) == int((h < 0).sum())
    to = oracle.prepare_textures(mo, log2n, tex_np, channels, "f32", hx.BUILD_MIPS | hx.MIRROR_BOUNDARY)
    ref_all = oracle.grad_to_pool_layout(to, oracle.lookup_grad(mo, to, (h, u, v, f), g.astype(np.float64)), 4)
    scale = np.abs(ref_all).max()
    assert np.abs(a - ref_all).max() <= 1e-5 * scale
    assert np.abs(b - ref_all).max() <= 1e-5 * scale
