"""csp_aggregate_noalloc against csp_aggregate, through the C ABI.

The allocation-free entry point serves callers that cannot allocate device
memory at aggregation time (stream capture, pre-reserved memory pools,
latency-bound loops).  It keeps its scratch in a fixed array shared by all
calls, so the test calls it twice in a row on different inputs and checks
each result against the allocating entry point.  This file is collected last
on purpose."""

import numpy as np
import pytest
import torch

import synthetic
from paper_1511_05174_gb300 import _binding as b
from paper_1511_05174_gb300.context import Context

pytestmark = pytest.mark.gpu


def _codes(w, ctx, seed):
    meas = torch.from_numpy(w.meas).cuda()
    Y = ctx.extract(meas)
    K = [int(k[0]) for k in w.K_levels]
    sup, coef, keff = ctx.solve(Y, "cross_scale", "fp32", K=K, Kmax=K[0])
    if seed:
        coef = coef * (1.0 + 0.25 * torch.randn_like(coef))
    return sup, coef.contiguous(), keff


def test_noalloc_aggregate_matches_aggregate_twice():
    w = synthetic.make_workload("bayer", H=64, W=64)
    ctx = Context(0)
    ctx.load_workload(w)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        sup, coef, keff = _codes(w, ctx, call)
        ref = ctx.aggregate(sup, coef, keff)
        out = torch.full_like(ref, float("nan"))
        b.csp_aggregate_noalloc(ctx._ctx, sup.data_ptr(), coef.data_ptr(), keff.data_ptr(), sup.shape[0],
                                sup.shape[1], out.data_ptr(), stream)
        torch.cuda.synchronize()
        r, o = ref.double().cpu().numpy(), out.double().cpu().numpy()
        scale = max(np.abs(r).max(), 1e-30)
        assert np.isfinite(o).all()
        assert np.abs(o - r).max() <= 1e-5 * scale, call


def test_noalloc_first_call_on_a_fresh_context_takes_no_device_memory():
    """Free device memory (cudaMemGetInfo) is the same before and after the
    entry point's first call on a freshly created context: the scratch array is
    reserved when the context is created, and the call itself allocates
    nothing."""
    w = synthetic.make_workload("bayer", H=48, W=48)
    ctx = Context(0)
    ctx.load_workload(w)
    sup, coef, keff = _codes(w, ctx, 0)
    ref = ctx.aggregate(sup, coef, keff)   # loads the aggregation kernels
    out = torch.full_like(ref, float("nan"))
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        b.csp_aggregate_noalloc(ctx._ctx, sup.data_ptr(), coef.data_ptr(), keff.data_ptr(), sup.shape[0],
                                sup.shape[1], out.data_ptr(), stream)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    assert torch.equal(out, ref)


@pytest.mark.parametrize("name,kw", [
    ("bayer", dict(H=64, W=72)),
    ("denoise", dict(H=64, W=72)),
    ("video", dict(H=48, W=40, T0=1024)),
    ("lightfield", dict(H=40, W=48, T0=2048)),
])
def test_fused_tile_aggregation_equals_two_pass(name, kw):
    """The fused shared-memory tile path, the two-pass path and the no-alloc
    entry point (two-pass on a fixed scratch): same arithmetic in the same
    order, so the images are bit-identical (ragged grids included)."""
    w = synthetic.make_workload(name, **kw)
    if name == "denoise":
        w.geometry.stride = 3
    ctx = Context(0)
    ctx.load_workload(w)
    stream = torch.cuda.current_stream().cuda_stream
    meas = torch.from_numpy(w.meas).cuda()
    Y = ctx.extract(meas)
    K = [int(np.max(k)) for k in w.K_levels]
    sup, coef, keff = ctx.solve(Y, "plain", "fp32", K=K[:1], Kmax=K[0])
    ctx.set_aggregate_path(2)
    ref = ctx.aggregate(sup, coef, keff)
    ctx.set_aggregate_path(1)
    two = ctx.aggregate(sup, coef, keff)
    out = torch.full_like(ref, float("nan"))
    b.csp_aggregate_noalloc(ctx._ctx, sup.data_ptr(), coef.data_ptr(), keff.data_ptr(), sup.shape[0],
                            sup.shape[1], out.data_ptr(), stream)
    torch.cuda.synchronize()
    assert torch.equal(ref, out) and torch.equal(two, out)
    with pytest.raises(b.CspError):
        ctx.set_aggregate_path(3)


def test_noalloc_rejects_oversized_batches():
    w = synthetic.make_workload("bayer")  # 64,009 patches x 192 > 4 Mi floats
    ctx = Context(0)
    ctx.load_workload(w)
    B = w.n_patches
    sup = torch.zeros((B, 8), dtype=torch.int32, device="cuda")
    coef = torch.zeros((B, 8), dtype=torch.float32, device="cuda")
    keff = torch.zeros((B,), dtype=torch.int8, device="cuda")
    img = torch.empty((3, 512, 512), dtype=torch.float32, device="cuda")
    with pytest.raises(b.CspError) as e:
        b.csp_aggregate_noalloc(ctx._ctx, sup.data_ptr(), coef.data_ptr(), keff.data_ptr(), B, 8, img.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert e.value.status == b.CSP_ERR_INVALID and "exceeds" in str(e.value)
