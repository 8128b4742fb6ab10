"""GPU path (through the C ABI) against the FP64 oracle on the same seeded
inputs.

Bar (FP32 path): support sets identical on >= 99.9 % of patches and, on those,
per-patch reconstruction D_|Omega alpha within 1e-4 relative L2 of the
oracle's; image PSNR within 0.05 dB.  Extraction is exact (a copy)."""

import numpy as np
import pytest
import torch

import oracle
import synthetic
from _gpu_util import budgets, compare, run_gpu

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4
MATCH = 0.999

SMALL = {
    # name: workload kwargs -- several proxy tiles (64 patches) and ragged patch grids
    "denoise": dict(name="denoise"),
    "denoise_ragged": dict(name="denoise", H=64, W=72),
    "bayer": dict(name="bayer", H=64, W=64),
    "lightfield": dict(name="lightfield", H=48, W=48, T0=2048),
    "video": dict(name="video", H=48, W=48, T0=1024),
    "inpaint": dict(name="inpaint", H=64, W=56, T0=512),
    "cs_dense": dict(name="cs_dense", H=64, W=72, T0=512),
    "rgb_identity": dict(name="bayer", H=48, W=48),   # Phi = I on RGB: M = 192 at the fine scale
}


def _workload(key, links="paper", **kw):
    spec = dict(SMALL[key])
    name = spec.pop("name")
    spec.update(kw)
    w = synthetic.make_workload(name, links=links, **spec)
    if key == "rgb_identity":
        rng = np.random.default_rng(9)
        w.sensing = synthetic.Sensing("identity")
        w.meas = (w.truth + w.sigma * rng.standard_normal(w.truth.shape)).astype(np.float32)
    if key == "denoise_ragged":
        w.geometry.stride = 3   # (72 - 8) % 3 != 0: clamped last origin on x
        B = w.n_patches
        w.K_levels = [np.full(B, int(k[0]), np.int32) for k in w.K_levels]
    return w


@pytest.mark.parametrize("key", [k for k in SMALL if k != "cs_dense"])
def test_extract_is_exact(key):
    w = _workload(key)
    g = run_gpu(w, "plain")
    np.testing.assert_array_equal(g["Y"], oracle.extract_patches(w).astype(np.float32))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("links", ["paper", "model"])
@pytest.mark.parametrize("key", list(SMALL))
def test_plain_parity(key, links, prec):
    """BF16: tensor-core proxy (tcgen05) with the top candidates re-scored in
    FP32 -- held to the same support bar as the FP32 path.  The model reading's
    fine atoms come in coherent sibling groups (they share their parent's
    structure)."""
    w = _workload(key, links=links)
    # video: per-patch Phi, the lifted proxy runs at dimension 512 (eight K blocks)
    g = run_gpu(w, "plain", prec)
    o, a, k, _ = oracle.plain_omp(w)
    rate, worst, bad = compare(w.dicts[0], g["sup"], g["coef"], g["keff"], o, a, k)
    assert rate >= MATCH, f"support mismatch on patches {bad[:10]}"
    assert worst <= REL_TOL


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("links", ["paper", "literal", "model"])
@pytest.mark.parametrize("key", list(SMALL))
def test_cross_scale_parity(key, links, prec):
    w = _workload(key, links=links)
    g = run_gpu(w, "cross_scale", prec)
    o, a, k, _ = oracle.cross_scale_omp(w)
    rate, worst, bad = compare(w.dicts[0], g["sup"], g["coef"], g["keff"], o, a, k)
    assert rate >= MATCH, f"support mismatch on patches {bad[:10]}"
    assert worst <= REL_TOL
    assert g["stats"]["overflow"] == 0


def test_dense_sensing_has_no_extraction():
    from paper_1511_05174_gb300 import _binding as b
    from paper_1511_05174_gb300.context import Context
    w = _workload("cs_dense")
    ctx = Context(0)
    ctx.load_workload(w)
    assert ctx.M == w.sensing.codes.shape[0]
    with pytest.raises(b.CspError) as e:
        ctx.extract(torch.zeros(64, 72, device="cuda"))
    assert e.value.status == b.CSP_ERR_UNSUPPORTED


@pytest.mark.parametrize("key", ["denoise", "bayer", "lightfield", "video", "inpaint", "cs_dense"])
def test_aggregate_matches_oracle(key):
    """Overlap-add of the GPU's own codes against the oracle's aggregation of
    the same codes."""
    w = _workload(key)
    g = run_gpu(w, "cross_scale")
    ref = oracle.aggregate(w, g["sup"], g["coef"].astype(np.float64), g["keff"])
    scale = max(np.abs(ref).max(), 1e-30)
    assert np.abs(g["img"] - ref).max() <= 1e-5 * scale


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("mode", ["plain", "cross_scale"])
def test_psnr_matches_oracle(mode, prec):
    w = _workload("bayer")
    g = run_gpu(w, mode, prec)
    o, a, k, _ = oracle.plain_omp(w) if mode == "plain" else oracle.cross_scale_omp(w)
    img_o = oracle.aggregate(w, o, a, k)
    assert abs(oracle.psnr(w.truth, g["img"]) - oracle.psnr(w.truth, img_o)) <= 0.05


@pytest.mark.parametrize("prec,form", [("fp32", 0), ("bf16", 1), ("bf16", 2), ("bf16", 3)])
def test_bayer_all_four_phases(prec, form):
    """Stride 1 puts patch origins on every RGGB phase: the patches of a phase
    are a non-identity subset of the grid, so every full-dictionary form runs
    with a permuted patch order (and the BF16 proxy with its sorted-position
    residual tile)."""
    from paper_1511_05174_gb300.context import Context
    w = synthetic.make_workload("bayer", H=40, W=40)
    w.geometry.stride = 1
    B = w.n_patches
    w.K_levels = [np.full(B, int(k[0]), np.int32) for k in w.K_levels]
    for mode, fn in (("plain", oracle.plain_omp), ("cross_scale", oracle.cross_scale_omp)):
        ctx = Context(0)
        ctx.set_top_level_form(form)
        g = run_gpu(w, mode, prec, ctx=ctx)
        o, a, k, _ = fn(w)
        rate, worst, bad = compare(w.dicts[0], g["sup"], g["coef"], g["keff"], o, a, k)
        assert rate >= MATCH and worst <= REL_TOL, (mode, bad[:10])


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("B,M,T,K", [(1000, 64, 320, 6), (999, 64, 300, 8), (257, 256, 8192, 12),
                                     (130, 128, 1000, 5), (64, 16, 64, 3)])
def test_independent_problems_nonunit_norms(B, M, T, K, prec):
    """Phi = I over independent problems with column norms in [0.5, 2] (the
    angle proxy divides by ||a_i||), noisy; ragged patch counts (tile 64/128)
    and atom counts (tile 128), M from 16 to 256."""
    from paper_1511_05174_gb300.context import Context
    A, Y, _ = synthetic.make_independent_problems(B, M, T, K, seed=3, sigma=0.05)
    ctx = Context(0)
    ctx.set_geometry(8, 8, (1, M // 64 if M >= 64 else 1), 8 if M >= 64 else 4, 8, [(1, 1, 1, 1)])
    ctx.set_sensing("identity")
    ctx.load_dictionary(0, A)
    sup, coef, keff = ctx.solve(torch.from_numpy(Y).cuda(), "plain", prec, K=[K], Kmax=K + 2)
    o, a, k, _ = oracle.omp_batch([A] * len(Y), Y, K)
    rate, worst, bad = compare(A, sup.cpu().numpy(), coef.cpu().numpy(), keff.cpu().numpy().astype(int), o, a, k)
    assert rate >= MATCH and worst <= REL_TOL, bad[:10]


@pytest.mark.parametrize("form", [1, 2, 3])
@pytest.mark.parametrize("B,M,T,K", [(1000, 64, 256, 6), (777, 64, 192, 5), (300, 16, 64, 3), (129, 32, 128, 8),
                                     (200, 128, 100, 7)])
def test_full_dictionary_forms_agree_with_oracle(B, M, T, K, form):
    """The fused full-dictionary kernel (form 2: every iteration of 128 patches
    in one CTA), the per-iteration kernels (form 1), BF16 proxy with FP32
    re-score, and the Gram form (form 3: correlation GEMM once, Gram-Schmidt
    iteration over every atom in FP32), against the oracle; ragged tiles
    (patches and atoms), per-patch budgets."""
    from paper_1511_05174_gb300.context import Context
    A, Y, _ = synthetic.make_independent_problems(B, M, T, K, seed=5, sigma=0.05)
    Kp = np.random.default_rng(6).integers(0, K + 1, size=B).astype(np.int8)
    ctx = Context(0)
    ctx.set_geometry(8, 8, (1, M // 64 if M >= 64 else M // 16), 8 if M >= 64 else 4, 8, [(1, 1, 1, 1)])
    ctx.set_sensing("identity")
    ctx.load_dictionary(0, A)
    ctx.set_top_level_form(form)
    ctx.profile(True)
    sup, coef, keff = ctx.solve(torch.from_numpy(Y).cuda(), "plain", "bf16", K=[K],
                                K_patch=[torch.from_numpy(Kp).cuda()], Kmax=K)
    prof = ctx.profile_read()
    assert ("omp_fused" in prof) == (form == 2 and T % 64 == 0 and M <= 64)
    assert ("full_gram" in prof) == (form == 3)
    o, a, k, _ = oracle.omp_batch([A] * len(Y), Y, [int(x) for x in Kp])
    rate, worst, bad = compare(A, sup.cpu().numpy(), coef.cpu().numpy(), keff.cpu().numpy().astype(int), o, a, k)
    assert rate >= MATCH and worst <= REL_TOL, bad[:10]


@pytest.mark.parametrize("H,stride,n_sample", [(512, 2, 300), (168, 1, 300)])
def test_fused_form_at_size(H, stride, n_sample):
    """Fused full-dictionary form forced on the Bayer coarse level (T 256, M 64,
    K 4), cross-scale: the 512x512 image (64,009 patches, one mosaic phase,
    two 128-patch tiles per CTA) and a stride-1 168x168 image (25,921 patches
    over the four phases in one launch); the oracle solves a seeded sample."""
    from paper_1511_05174_gb300.context import Context
    w = synthetic.make_workload("bayer", H=H, W=H)
    w.geometry.stride = stride
    B = w.n_patches
    w.K_levels = [np.full(B, int(k[0]), np.int32) for k in w.K_levels]
    sample = np.sort(np.random.default_rng(1).choice(B, n_sample, replace=False))
    ctx = Context(0)
    ctx.load_workload(w)
    Yd = ctx.extract(torch.from_numpy(w.meas).cuda())
    K, K_patch, Kmax = budgets(w, "cross_scale")
    ctx.set_top_level_form(2)
    ctx.set_pipeline(False)
    ctx.profile(True)
    sup, coef, keff = ctx.solve(Yd, "cross_scale", "bf16", K=K, K_patch=K_patch, Kmax=Kmax)
    prof = ctx.profile_read()
    assert prof["omp_fused"][0] == 1  # one launch for every phase
    o, a, k, _ = oracle.cross_scale_omp(w, Y=oracle.extract_patches(w), patches=sample)
    rate, worst, bad = compare(w.dicts[0], sup.cpu().numpy()[sample], coef.cpu().numpy()[sample],
                               keff.cpu().numpy().astype(np.int64)[sample], o, a, k)
    assert rate >= MATCH and worst <= REL_TOL, sample[bad[:10]]


def test_fused_form_rejects_dependent_atom():
    """Fused form: a_2 = a_0 + a_1 exactly (integer atoms, the other 61 atoms
    zero and never eligible); the FP64 pivot test rejects a_2, k_eff = 2 and
    the coefficients are the least squares ones, as in the oracle."""
    from paper_1511_05174_gb300.context import Context
    rng = np.random.default_rng(14)
    A = np.zeros((64, 64), np.float32)
    A[:2] = rng.integers(-3, 4, size=(2, 64))
    A[2] = A[0] + A[1]
    Y = np.stack([A[0] + 0.5 * A[1] + 0.01 * rng.standard_normal(64) for _ in range(40)]).astype(np.float32)
    ctx = Context(0)
    ctx.set_geometry(8, 8, (1, 1), 8, 8, [(1, 1, 1, 1)])
    ctx.set_sensing("identity")
    ctx.load_dictionary(0, A)
    ctx.set_top_level_form(2)
    sup, coef, keff = ctx.solve(torch.from_numpy(Y).cuda(), "plain", "bf16", K=[3], Kmax=3)
    o, a, k, _ = oracle.omp_batch([A[:3]] * len(Y), Y, 3)
    assert np.all(k == 2) and np.all(keff.cpu().numpy() == 2)
    assert ctx.stats()["fp64_fallbacks"] >= 1
    rate, worst, bad = compare(A[:3], sup.cpu().numpy(), coef.cpu().numpy(), keff.cpu().numpy().astype(int), o, a, k)
    assert rate == 1.0 and worst <= REL_TOL


def test_degenerate_inputs():
    """Zero measurements (k_eff = 0), duplicate atoms (dependence), a zero
    atom (never chosen) and K = 1."""
    from paper_1511_05174_gb300.context import Context
    A, Y, _ = synthetic.make_independent_problems(300, 64, 128, 4, seed=5, sigma=0.01)
    A = A.copy()
    A[7] = 0.0
    A[9] = A[3]
    Y = Y.copy()
    Y[::10] = 0.0
    # a measurement exactly in the span of {3, 9}: 9 duplicates 3, so OMP picks 3 then must not add 9
    Y[1] = 2.0 * A[3]
    ctx = Context(0)
    ctx.set_geometry(8, 8, (1, 1), 8, 8, [(1, 1, 1, 1)])
    ctx.set_sensing("identity")
    ctx.load_dictionary(0, A)
    for K in (1, 4, 10):
        sup, coef, keff = ctx.solve(torch.from_numpy(Y).cuda(), "plain", "fp32", K=[K], Kmax=K)
        s, c, kk = sup.cpu().numpy(), coef.cpu().numpy(), keff.cpu().numpy().astype(int)
        o, a, k, _ = oracle.omp_batch([A] * len(Y), Y, K)
        assert np.all(kk[::10] == 0) and np.all(k[::10] == 0)
        assert not np.any(s == 7)
        assert np.all(np.isfinite(c))
        assert s[1, 0] == 3 and kk[1] == 1
        rate, worst, bad = compare(A, s, c, kk, o, a, k)
        assert rate >= MATCH and worst <= REL_TOL, (K, bad[:10])


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_maximum_sparsity_budget(prec):
    """K = CSP_MAX_K = 32 on noiseless 32-sparse problems (M = 128, T = 256):
    the largest factor, the longest chains, ragged patch tile (200)."""
    from paper_1511_05174_gb300.context import Context
    A, Y, _ = synthetic.make_independent_problems(200, 128, 256, 32, seed=9, sigma=0.0, unit_norm=True)
    ctx = Context(0)
    ctx.set_geometry(8, 8, (1, 2), 8, 8, [(1, 1, 1, 1)])
    ctx.set_sensing("identity")
    ctx.load_dictionary(0, A)
    sup, coef, keff = ctx.solve(torch.from_numpy(Y).cuda(), "plain", prec, K=[32], Kmax=32)
    o, a, k, _ = oracle.omp_batch([A] * len(Y), Y, 32)
    rate, worst, bad = compare(A, sup.cpu().numpy(), coef.cpu().numpy(), keff.cpu().numpy().astype(int), o, a, k)
    assert rate >= MATCH and worst <= REL_TOL, bad[:10]


def test_empty_batch():
    """B = 0: nothing to solve, nothing written, no error."""
    from paper_1511_05174_gb300.context import Context
    A, _, _ = synthetic.make_independent_problems(1, 64, 128, 4, seed=1)
    ctx = Context(0)
    ctx.set_geometry(8, 8, (1, 1), 8, 8, [(1, 1, 1, 1)])
    ctx.set_sensing("identity")
    ctx.load_dictionary(0, A)
    for prec in ("fp32", "bf16"):
        sup, coef, keff = ctx.solve(torch.zeros((0, 64), device="cuda"), "plain", prec, K=[4], Kmax=4)
        torch.cuda.synchronize()
        assert sup.shape == (0, 4) and keff.shape == (0,)
        assert ctx.stats()["patches"] == 0


def test_per_patch_budgets_lightfield():
    """K drawn per patch in [8, 20] (and ceil(K/2), ceil(K/4) at coarser scales)."""
    w = _workload("lightfield")
    assert len(np.unique(w.K_levels[0])) > 3
    for mode, fn in (("plain", oracle.plain_omp), ("cross_scale", oracle.cross_scale_omp)):
        g = run_gpu(w, mode)
        o, a, k, _ = fn(w)
        assert np.all(g["keff"] <= w.K_levels[0])
        rate, worst, bad = compare(w.dicts[0], g["sup"], g["coef"], g["keff"], o, a, k)
        assert rate >= MATCH and worst <= REL_TOL, (mode, bad[:10])


def test_deterministic():
    w = _workload("bayer")
    g1 = run_gpu(w, "cross_scale")
    g2 = run_gpu(w, "cross_scale")
    for key in ("sup", "coef", "keff", "img"):
        np.testing.assert_array_equal(g1[key], g2[key])


@pytest.mark.parametrize("name,prec,n_sample", [
    ("bayer", "fp32", 300), ("bayer", "bf16", 300), ("video", "bf16", 120), ("lightfield", "bf16", 60),
    ("inpaint", "bf16", 300),
])
def test_full_size_sampled(name, prec, n_sample):
    """Full-size workload in the benchmark's launch configuration (the
    autotuner picks the restricted variant and the full-dictionary form first);
    the oracle solves a seeded sample of patches, plain and cross-scale."""
    from paper_1511_05174_gb300.context import Context
    w = synthetic.make_workload(name)
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(w.n_patches, n_sample, replace=False))
    Y = oracle.extract_patches(w)
    ctx = Context(0)
    ctx.load_workload(w)
    Yd = ctx.extract(torch.from_numpy(w.meas).cuda())
    Kc, K_patch, Kmax = budgets(w, "cross_scale")
    ctx.autotune(Yd, "cross_scale", prec, K=Kc, K_patch=K_patch, Kmax=Kmax)
    for mode, fn in (("plain", oracle.plain_omp), ("cross_scale", oracle.cross_scale_omp)):
        K, K_patch, Kmax = budgets(w, mode)
        sup, coef, keff = ctx.solve(Yd, mode, prec, K=K, K_patch=K_patch, Kmax=Kmax)
        o, a, k, _ = fn(w, Y=Y, patches=sample)
        rate, worst, bad = compare(w.dicts[0], sup.cpu().numpy()[sample], coef.cpu().numpy()[sample],
                                   keff.cpu().numpy().astype(np.int64)[sample], o, a, k)
        assert rate >= MATCH and worst <= REL_TOL, (mode, sample[bad[:10]])


def test_invalid_arguments_raise():
    from paper_1511_05174_gb300 import _binding as b
    from paper_1511_05174_gb300.context import Context
    w = _workload("denoise")
    ctx = Context(0)
    ctx.load_workload(w)
    bad = w.parents[0].copy()
    bad[0] = 10_000
    with pytest.raises(b.CspError) as e:
        ctx.load_links(0, bad)
    assert e.value.status == b.CSP_ERR_INVALID
    Y = torch.zeros((w.n_patches, 64), device="cuda")
    with pytest.raises(b.CspError):
        ctx.solve(Y, "plain", "fp32", K=[40], Kmax=40)
    small = Context(0, mem_budget_bytes=4096)
    small.set_geometry(64, 64, (1, 1), 8, 8, [(1, 1, 1, 1)])
    small.set_sensing("identity")
    with pytest.raises(b.CspError) as e:
        small.load_dictionary(0, w.dicts[0])
    assert e.value.status == b.CSP_ERR_OOM


def test_exactly_dependent_atom_ends_the_patch():
    """Integer atoms make a_2 = a_0 + a_1 exact in float32: after a_0 and a_1
    the only eligible atom depends on them, the FP64 pivot test rejects it and
    k_eff = 2 (as the oracle's QR pivot does)."""
    from paper_1511_05174_gb300.context import Context
    rng = np.random.default_rng(12)
    A = rng.integers(-3, 4, size=(3, 64)).astype(np.float32)
    A[2] = A[0] + A[1]
    Y = np.stack([A[0] + 0.5 * A[1] + 0.01 * rng.standard_normal(64) for _ in range(40)]).astype(np.float32)
    ctx = Context(0)
    ctx.set_geometry(8, 8, (1, 1), 8, 8, [(1, 1, 1, 1)])
    ctx.set_sensing("identity")
    ctx.load_dictionary(0, A)
    sup, coef, keff = ctx.solve(torch.from_numpy(Y).cuda(), "plain", "fp32", K=[3], Kmax=3)
    o, a, k, _ = oracle.omp_batch([A] * len(Y), Y, 3)
    assert np.all(k == 2)
    assert np.all(keff.cpu().numpy() == 2)
    assert ctx.stats()["fp64_fallbacks"] >= 1
    rate, worst, bad = compare(A, sup.cpu().numpy(), coef.cpu().numpy(), keff.cpu().numpy().astype(int), o, a, k)
    assert rate == 1.0 and worst <= REL_TOL


@pytest.mark.parametrize("variant", list(range(14)))
def test_restricted_dependent_candidate_falls_back_to_fp64(variant):
    """Fine step of Algorithm 2 whose candidate set holds an exactly dependent
    atom (a_2 = a_0 + a_1, integer atoms): every restricted variant rejects it
    through the FP64 pivot test, k_eff = 2, and the coefficients are the least
    squares ones, as in the oracle (one coarse atom whose children are all
    fine atoms: cross-scale OMP equals plain OMP here)."""
    from paper_1511_05174_gb300.context import Context
    rng = np.random.default_rng(13)
    A = rng.integers(-3, 4, size=(3, 64)).astype(np.float32)
    A[2] = A[0] + A[1]
    Y = np.stack([A[0] + 0.5 * A[1] + 0.01 * rng.standard_normal(64) for _ in range(40)]).astype(np.float32)
    coarse = A[:1].reshape(1, 8, 8)
    coarse = coarse.reshape(1, 4, 2, 4, 2).mean(axis=(2, 4)).reshape(1, 16).astype(np.float32)
    ctx = Context(0)
    ctx.set_geometry(8, 8, (1, 1), 8, 8, [(1, 1, 1, 1), (1, 1, 2, 2)])
    ctx.set_sensing("identity")
    ctx.load_dictionary(0, A)
    ctx.load_dictionary(1, coarse)
    ctx.load_links(0, np.zeros(3, np.int32))
    ctx.set_kernel_variant(variant)
    sup, coef, keff = ctx.solve(torch.from_numpy(Y).cuda(), "cross_scale", "fp32", K=[3, 1], Kmax=3)
    o, a, k, _ = oracle.omp_batch([A] * len(Y), Y, 3)
    assert np.all(k == 2)
    assert np.all(keff.cpu().numpy() == 2)
    assert ctx.stats()["fp64_fallbacks"] >= 1
    rate, worst, bad = compare(A, sup.cpu().numpy(), coef.cpu().numpy(), keff.cpu().numpy().astype(int), o, a, k)
    assert rate == 1.0 and worst <= REL_TOL


@pytest.mark.parametrize("variant", [0, 2, 6, 8, 12])
def test_per_pixel_dependent_candidate_falls_back_to_fp64(variant):
    """The dependent-atom case above on per-pixel Phi: a one-frame coded exposure
    whose codes are all 1 (so every patch's effective rows are the atoms
    themselves), 40 patches in one row of the image.  The restricted level takes
    each patch's candidate rows and, for variants >= 2, their per-patch Gram
    blocks; the FP64 rebuild reads the rows of the patch's own slots.  k_eff = 2
    and least-squares coefficients, as in the oracle."""
    from paper_1511_05174_gb300.context import Context
    rng = np.random.default_rng(13)
    A = rng.integers(-3, 4, size=(3, 64)).astype(np.float32)
    A[2] = A[0] + A[1]
    Y = np.stack([A[0] + 0.5 * A[1] + 0.01 * rng.standard_normal(64) for _ in range(40)]).astype(np.float32)
    coarse = A[:1].reshape(1, 4, 2, 4, 2).mean(axis=(2, 4)).reshape(1, 16).astype(np.float32)
    ctx = Context(0)
    ctx.set_geometry(8, 320, (1, 1), 8, 8, [(1, 1, 1, 1), (1, 1, 2, 2)])
    ctx.set_sensing("coded_exposure", np.ones((1, 8, 320), np.uint8))
    ctx.load_dictionary(0, A)
    ctx.load_dictionary(1, coarse)
    ctx.load_links(0, np.zeros(3, np.int32))
    ctx.set_kernel_variant(variant)
    sup, coef, keff = ctx.solve(torch.from_numpy(Y).cuda(), "cross_scale", "fp32", K=[3, 1], Kmax=3)
    o, a, k, _ = oracle.omp_batch([A] * len(Y), Y, 3)
    assert np.all(k == 2)
    assert np.all(keff.cpu().numpy() == 2)
    assert ctx.stats()["fp64_fallbacks"] >= 1
    rate, worst, bad = compare(A, sup.cpu().numpy(), coef.cpu().numpy(), keff.cpu().numpy().astype(int), o, a, k)
    assert rate == 1.0 and worst <= REL_TOL


@pytest.mark.parametrize("variant", list(range(14)))
@pytest.mark.parametrize("key", ["bayer", "lightfield", "denoise_ragged", "video", "rgb_identity"])
def test_restricted_variants_agree_with_oracle(key, variant):
    """Every restricted-solver variant the autotuner may pick meets the parity
    bar: L2-cooperative (0), shared-memory staged (1), Gram-matrix proxy with
    narrow, middle and wide lane groups (2, 3, 4), its Gram-Schmidt form (5, 6, 7),
    the register forms (8-13).  On the per-pixel-Phi video workload variants 2-13
    run the Gram-Schmidt form on the per-patch Gram blocks of the candidate rows."""
    from paper_1511_05174_gb300.context import Context
    w = _workload(key)
    o, a, k, _ = oracle.cross_scale_omp(w)
    ctx = Context(0)
    ctx.load_workload(w)
    ctx.set_kernel_variant(variant)
    Y = ctx.extract(torch.from_numpy(w.meas).cuda())
    K, K_patch, Kmax = budgets(w, "cross_scale")
    sup, coef, keff = ctx.solve(Y, "cross_scale", "fp32", K=K, K_patch=K_patch, Kmax=Kmax)
    rate, worst, bad = compare(w.dicts[0], sup.cpu().numpy(), coef.cpu().numpy(),
                               keff.cpu().numpy().astype(np.int64), o, a, k)
    assert rate >= MATCH and worst <= REL_TOL, bad[:10]


def test_expired_device_wait_is_reported_and_context_recovers():
    """Failure detection without a fault: with the test hook the tensor-core
    proxy loads no atom tiles, its bounded wait expires, the solve reports
    CSP_ERR_TIMEOUT through the statistics; afterwards the same context solves
    correctly."""
    from paper_1511_05174_gb300 import _binding as b
    from paper_1511_05174_gb300.context import Context
    w = _workload("bayer")
    ctx = Context(0)
    ctx.load_workload(w)
    ctx.set_top_level_form(1)
    Y = ctx.extract(torch.from_numpy(w.meas).cuda())
    K, K_patch, Kmax = budgets(w, "cross_scale")
    ctx.set_wait_test(True)
    ctx.solve(Y, "cross_scale", "bf16", K=K, K_patch=K_patch, Kmax=Kmax)
    torch.cuda.synchronize()
    with pytest.raises(b.CspError) as e:
        ctx.stats()
    assert e.value.status == b.CSP_ERR_TIMEOUT
    ctx.set_wait_test(False)
    sup, coef, keff = ctx.solve(Y, "cross_scale", "bf16", K=K, K_patch=K_patch, Kmax=Kmax)
    st = ctx.stats()
    assert st["patches"] == w.n_patches
    o, a, k, _ = oracle.cross_scale_omp(w)
    rate, worst, bad = compare(w.dicts[0], sup.cpu().numpy(), coef.cpu().numpy(),
                               keff.cpu().numpy().astype(np.int64), o, a, k)
    assert rate >= MATCH and worst <= REL_TOL


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_graph_mode_replays_identical_results(prec):
    """Graph mode: the first solve runs and records, the next identical calls
    replay the CUDA graph; new measurement values in the same buffer, another
    kernel variant or another batch are handled; results equal graph-off ones."""
    from paper_1511_05174_gb300.context import Context
    w = _workload("bayer")
    w2 = synthetic.make_workload("bayer", H=64, W=64, seed=7, dict_seed=0)
    ref = Context(0)
    ref.load_workload(w)
    ctx = Context(0)
    ctx.load_workload(w)
    ctx.set_graph_mode(True)
    K, K_patch, Kmax = budgets(w, "cross_scale")
    Y = ctx.extract(torch.from_numpy(w.meas).cuda())
    Yr = ref.extract(torch.from_numpy(w.meas).cuda())
    outs = (torch.empty((w.n_patches, Kmax), dtype=torch.int32, device="cuda"),
            torch.empty((w.n_patches, Kmax), dtype=torch.float32, device="cuda"),
            torch.empty((w.n_patches,), dtype=torch.int8, device="cuda"))

    def same(meas, variant):
        ctx.set_kernel_variant(variant)
        ref.set_kernel_variant(variant)
        ctx.extract(torch.from_numpy(meas).cuda(), Y)
        ref.extract(torch.from_numpy(meas).cuda(), Yr)
        for _ in range(3):  # record, then replay twice
            for t in outs:
                t.fill_(0)
            ctx.solve(Y, "cross_scale", prec, K=K, K_patch=K_patch, Kmax=Kmax, out=outs)
            r = ref.solve(Yr, "cross_scale", prec, K=K, K_patch=K_patch, Kmax=Kmax)
            torch.cuda.synchronize()
            assert all(torch.equal(a, b) for a, b in zip(outs, r))
        assert ctx.stats()["patches"] == w.n_patches

    same(w.meas, 2)
    same(w2.meas, 2)  # same buffers, new contents: replayed
    same(w2.meas, 6)  # another variant: recorded again
    ctx.set_graph_mode(False)
    same(w.meas, 0)


def test_autotune_picks_a_variant():
    from paper_1511_05174_gb300.context import Context
    w = _workload("bayer")
    ctx = Context(0)
    ctx.load_workload(w)
    Y = ctx.extract(torch.from_numpy(w.meas).cuda())
    K, K_patch, Kmax = budgets(w, "cross_scale")
    r = ctx.autotune(Y, "cross_scale", "bf16", K=K, K_patch=K_patch, Kmax=Kmax)
    assert r["restricted_variant"] in range(14) and all(t > 0 for t in r["ms"])
    assert r["ms"][r["restricted_variant"]] == min(r["ms"])
    # the BF16 Bayer coarse level (T = 256, M = 64, K = 4) has all three full-dictionary forms
    r2 = ctx.autotune(Y, "cross_scale", "bf16", K=K, K_patch=K_patch, Kmax=Kmax)
    assert r2["top_level_form"] in (1, 2, 3) and all(t > 0 for t in r2["ms_top"])  # form 3 applies too
    assert r2["ms_top"][r2["top_level_form"] - 1] == min(r2["ms_top"])


def test_pipelined_solve_equals_one_stream():
    """The pipelined cross-scale solve (first wave of the fused kernel's patches
    down the scales on a second stream) gives the one-stream results exactly,
    also when recorded in a CUDA graph and replayed."""
    from paper_1511_05174_gb300.context import Context
    w = synthetic.make_workload("bayer")
    ctx = Context(0)
    ctx.load_workload(w)
    Yd = ctx.extract(torch.from_numpy(w.meas).cuda())
    K, K_patch, Kmax = budgets(w, "cross_scale")
    ctx.set_top_level_form(2)
    ctx.set_pipeline(False)
    ref = [t.cpu().numpy() for t in ctx.solve(Yd, "cross_scale", "bf16", K=K, K_patch=K_patch, Kmax=Kmax)]
    ctx.set_pipeline(True)
    ctx.profile_read(reset=True)
    ctx.profile(True)
    ctx.solve(Yd, "cross_scale", "bf16", K=K, K_patch=K_patch, Kmax=Kmax)
    prof = ctx.profile_read(reset=True)
    ctx.profile(False)
    assert prof["omp_fused"][0] == 2 and prof["restricted"][0] == 2  # two chunks
    ctx.set_graph_mode(True)
    B = Yd.shape[0]
    out = (torch.empty((B, Kmax), dtype=torch.int32, device="cuda"),
           torch.empty((B, Kmax), dtype=torch.float32, device="cuda"),
           torch.empty((B,), dtype=torch.int8, device="cuda"))
    for _ in range(3):  # run and record, then two replays
        for t in out:
            t.fill_(-7)
        ctx.solve(Yd, "cross_scale", "bf16", K=K, K_patch=K_patch, Kmax=Kmax, out=out)
        torch.cuda.synchronize()
        for a, t in zip(ref, out):
            assert np.array_equal(a, t.cpu().numpy())
    ctx.set_graph_mode(False)


@pytest.mark.parametrize("key,mode,prec,variant,form", [
    ("bayer", "cross_scale", "bf16", 6, 2),   # finest level synthesizes x_hat itself
    ("bayer", "cross_scale", "bf16", 0, 1),   # separate synthesis pass
    ("bayer", "plain", "fp32", 6, 1),
    ("denoise_ragged", "cross_scale", "fp32", 5, 1),
    ("inpaint", "cross_scale", "bf16", 6, 1),  # per-pixel Phi: no Gram variants
])
def test_reconstruct_equals_three_calls(key, mode, prec, variant, form):
    """csp_reconstruct (device buffers, one call) gives the image of
    extract + solve + aggregate exactly, also replayed from its CUDA graph."""
    from paper_1511_05174_gb300.context import Context
    w = _workload(key)
    ctx = Context(0)
    ctx.load_workload(w)
    ctx.set_kernel_variant(variant)
    ctx.set_top_level_form(form)
    meas = torch.from_numpy(np.ascontiguousarray(w.meas)).cuda()
    K, K_patch, Kmax = budgets(w, mode)
    assert K_patch is None
    Y = ctx.extract(meas)
    sup, coef, keff = ctx.solve(Y, mode, prec, K=K, Kmax=Kmax)
    ref = ctx.aggregate(sup, coef, keff).cpu().numpy()
    img = torch.full_like(torch.from_numpy(ref).cuda(), -3.0)
    ctx.reconstruct(meas, img, mode, prec, K=K, Kmax=Kmax)
    torch.cuda.synchronize()
    assert np.array_equal(img.cpu().numpy(), ref)
    ctx.set_graph_mode(True)
    for _ in range(3):  # record, then replay
        img.fill_(-3.0)
        ctx.reconstruct(meas, img, mode, prec, K=K, Kmax=Kmax)
        torch.cuda.synchronize()
        assert np.array_equal(img.cpu().numpy(), ref)
    host = np.zeros_like(ref)
    ctx.reconstruct_host(np.ascontiguousarray(w.meas), host, mode, prec, K=K, Kmax=Kmax)
    assert np.array_equal(host, ref)
    ctx.set_graph_mode(False)


def test_reconstruct_at_size_pipelined():
    """The 512x512 Bayer image through csp_reconstruct with the fused coarse
    level, the two-stream pipeline and the fused synthesis, graph-replayed:
    the image of the separate calls on one stream."""
    from paper_1511_05174_gb300.context import Context
    w = synthetic.make_workload("bayer")
    ctx = Context(0)
    ctx.load_workload(w)
    ctx.set_kernel_variant(6)
    ctx.set_top_level_form(2)
    meas = torch.from_numpy(np.ascontiguousarray(w.meas)).cuda()
    K, _, Kmax = budgets(w, "cross_scale")
    ctx.set_pipeline(False)
    Y = ctx.extract(meas)
    sup, coef, keff = ctx.solve(Y, "cross_scale", "bf16", K=K, Kmax=Kmax)
    ref = ctx.aggregate(sup, coef, keff).cpu().numpy()
    ctx.set_pipeline(True)
    ctx.set_graph_mode(True)
    img = torch.empty_like(torch.from_numpy(ref).cuda())
    for _ in range(3):
        img.fill_(-3.0)
        ctx.reconstruct(meas, img, "cross_scale", "bf16", K=K, Kmax=Kmax)
        torch.cuda.synchronize()
        assert np.array_equal(img.cpu().numpy(), ref)
    # page-locked host buffers: the copies are recorded in the graph as well
    meas_h = torch.from_numpy(np.ascontiguousarray(w.meas)).pin_memory()
    img_h = torch.empty(ref.shape, dtype=torch.float32).pin_memory()
    for _ in range(3):
        img_h.fill_(-3.0)
        ctx.reconstruct_host(meas_h, img_h, "cross_scale", "bf16", K=K, Kmax=Kmax)
        assert np.array_equal(img_h.numpy(), ref)
    assert ctx.stats()["synthesized"]
    ctx.set_graph_mode(False)


@pytest.mark.parametrize("Q,prec", [(2, "fp32"), (8, "bf16"), (16, "fp32")])
def test_cross_scale_other_link_sizes(Q, prec):
    """Children per coarse atom Q = 2, 8, 16 (coarse dictionary of T/Q atoms,
    uneven child counts), Bayer 64x64: supports and coefficients against the
    oracle, and through csp_reconstruct the oracle's image."""
    w = synthetic.make_workload("bayer", H=64, W=64, Q=Q)
    g = run_gpu(w, "cross_scale", prec)
    o, a, k, _ = oracle.cross_scale_omp(w)
    rate, worst, bad = compare(w.dicts[0], g["sup"], g["coef"], g["keff"], o, a, k)
    assert rate >= MATCH and worst <= REL_TOL, bad[:10]
    img_o = oracle.aggregate(w, o, a, k)
    assert abs(oracle.psnr(w.truth, g["img"]) - oracle.psnr(w.truth, img_o)) <= 0.05


@pytest.mark.parametrize("variant", [8, 9, 10, 11, 12, 13])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("key", ["bayer", "denoise", "denoise_ragged", "cs_dense", "rgb_identity"])
def test_register_variants_on_model_reading(key, prec, variant):
    """Restricted variants 8-13 (candidates' state in registers, 8, 16 and 4
    lanes per patch, iteration loop unrolled; 11-13 with each patch's Gram
    block staged in shared memory) on the model reading, where
    every candidate set fits them (|f(Omega)| = 4 K_low, K <= 8): supports and
    coefficients against the oracle, and csp_reconstruct (which then synthesizes
    x_hat in the same kernel) equal to extract + solve + aggregate, bit for bit."""
    from paper_1511_05174_gb300.context import Context
    w = _workload(key, links="model")
    assert max(int(np.max(k)) for k in w.K_levels) <= 8
    ctx = Context(0)
    ctx.load_workload(w)
    ctx.set_kernel_variant(variant)
    meas = torch.from_numpy(np.ascontiguousarray(w.meas)).cuda()
    Y = meas.contiguous() if w.sensing.kind == "dense" else ctx.extract(meas)
    K, K_patch, Kmax = budgets(w, "cross_scale")
    sup, coef, keff = ctx.solve(Y, "cross_scale", prec, K=K, K_patch=K_patch, Kmax=Kmax)
    o, a, k, _ = oracle.cross_scale_omp(w)
    rate, worst, bad = compare(w.dicts[0], sup.cpu().numpy(), coef.cpu().numpy(),
                               keff.cpu().numpy().astype(np.int64), o, a, k)
    assert rate >= MATCH and worst <= REL_TOL, bad[:10]
    assert ctx.stats()["overflow"] == 0
    if w.sensing.kind == "dense" or K_patch is not None:
        return
    ref = ctx.aggregate(sup, coef, keff).cpu().numpy()
    img = torch.full_like(torch.from_numpy(ref).cuda(), -3.0)
    ctx.reconstruct(meas, img, "cross_scale", prec, K=K, Kmax=Kmax)
    torch.cuda.synchronize()
    assert ctx.stats()["synthesized"]
    assert np.array_equal(img.cpu().numpy(), ref)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("key,links", [("bayer", "model"), ("bayer", "paper"), ("denoise", "model"),
                                       ("rgb_identity", "model"), ("cs_dense", "model"), ("denoise_ragged", "paper")])
def test_gram_form_of_the_coarse_level(key, links, prec):
    """Form 3 (Gram form) at the coarsest level of Algorithm 2: supports and
    coefficients against the oracle, and csp_reconstruct in graph mode equal to
    the three calls."""
    from paper_1511_05174_gb300.context import Context
    w = _workload(key, links=links)
    ctx = Context(0)
    ctx.load_workload(w)
    ctx.set_top_level_form(3)
    ctx.profile(True)
    meas = torch.from_numpy(np.ascontiguousarray(w.meas)).cuda()
    Y = meas.contiguous() if w.sensing.kind == "dense" else ctx.extract(meas)
    K, K_patch, Kmax = budgets(w, "cross_scale")
    sup, coef, keff = ctx.solve(Y, "cross_scale", prec, K=K, K_patch=K_patch, Kmax=Kmax)
    assert "full_gram" in ctx.profile_read()
    o, a, k, _ = oracle.cross_scale_omp(w)
    rate, worst, bad = compare(w.dicts[0], sup.cpu().numpy(), coef.cpu().numpy(),
                               keff.cpu().numpy().astype(np.int64), o, a, k)
    assert rate >= MATCH and worst <= REL_TOL, bad[:10]
    if w.sensing.kind == "dense" or K_patch is not None:
        return
    ref = ctx.aggregate(sup, coef, keff).cpu().numpy()
    img = torch.full_like(torch.from_numpy(ref).cuda(), -3.0)
    ctx.set_graph_mode(True)
    for _ in range(2):
        img.fill_(-3.0)
        ctx.reconstruct(meas, img, "cross_scale", prec, K=K, Kmax=Kmax)
        torch.cuda.synchronize()
        assert np.array_equal(img.cpu().numpy(), ref)
    ctx.set_graph_mode(False)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("variant", [2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("links", ["paper", "model"])
def test_work_order_sorted_queue_equals_static(links, variant, prec):
    """Per-patch budgets K in [8, 20] (light field): with the work order (patches
    sorted by budget, restricted levels on persistent warps fed by a work queue)
    every patch's result equals the static grid's bit for bit, and both meet
    the oracle; also recorded in a CUDA graph and replayed.  BF16 runs the
    full-dictionary level's tensor-core proxy on the sorted-position residual
    tile."""
    from paper_1511_05174_gb300.context import Context
    w = _workload("lightfield", links=links)
    K, K_patch, Kmax = budgets(w, "cross_scale")
    assert K_patch is not None
    ctx = Context(0)
    ctx.load_workload(w)
    ctx.set_kernel_variant(variant)
    Y = ctx.extract(torch.from_numpy(np.ascontiguousarray(w.meas)).cuda())
    ref = [t.cpu().numpy() for t in ctx.solve(Y, "cross_scale", prec, K=K, K_patch=K_patch, Kmax=Kmax)]
    ctx.set_work_order(1)
    ctx.set_graph_mode(True)
    for _ in range(3):
        got = [t.cpu().numpy() for t in ctx.solve(Y, "cross_scale", prec, K=K, K_patch=K_patch, Kmax=Kmax)]
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)
    ctx.set_graph_mode(False)
    o, a, k, _ = oracle.cross_scale_omp(w)
    rate, worst, bad = compare(w.dicts[0], got[0], got[1], got[2].astype(np.int64), o, a, k)
    assert rate >= MATCH and worst <= REL_TOL, bad[:10]
