"""The allocation-free unfused entry point (fkl_execute_batch_unfused_static).

Some callers cannot call cudaMalloc -- a host framework that owns every
device allocation under a fixed budget, or a latency-critical loop that must
not take cudaMalloc's implicit device synchronisation. For them the library
runs its unfused one-kernel-per-op form on a static device array instead of a
caller workspace. This file checks, through the C ABI, that two calls in a row
give the same output as the workspace-taking entry point, and that a batch
too large for the static array is refused before any work is enqueued.

It sits in a file of its own that pytest collects last, so a run that stops
at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2508_07071_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2508_07071_gb300 import build
    build.build()
    from paper_2508_07071_gb300 import fkl
    return fkl


def _with_workspace(F, p, ins, rois, out):
    nbytes = F.fkl_unfused_workspace_bytes(p.handle, ins, rois, out)
    ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda")
    F.fkl_execute_batch_unfused(p.handle, ins, rois, out, ws.data_ptr(), nbytes)
    torch.cuda.synchronize()


def test_static_scratch_matches_workspace_form_twice_in_a_row(F):
    from paper_2508_07071_gb300 import workloads as W

    # NV12 letterbox to bf16: 2 x 11 MB of intermediates per frame
    p = F.Pipeline(W.nv12_letterbox_chain(F.FKL_BF16))
    for call, seed in enumerate((11, 12)):
        frames = torch.from_numpy(synth.nv12_frames(seed, 2, 720, 1280)).cuda()
        ins = [F.as_fkl(frames[i], F.FKL_LAYOUT_NV12) for i in range(2)]
        want = torch.zeros((2, 3, 640, 640), dtype=torch.bfloat16, device="cuda")
        got = torch.full((2, 3, 640, 640), float("nan"), dtype=torch.bfloat16, device="cuda")
        _with_workspace(F, p, ins, None, F.as_fkl(want, F.FKL_LAYOUT_NCHW))
        F.fkl_execute_batch_unfused_static(p.handle, ins, None, F.as_fkl(got, F.FKL_LAYOUT_NCHW))
        torch.cuda.synchronize()
        assert torch.equal(got.view(torch.uint8), want.view(torch.uint8)), f"call {call}"

    # crops of a packed frame, normalised to float32
    p = F.Pipeline(W.normalize_chain(128, 64))
    frame = torch.from_numpy(synth.packed_image(1, 720, 1280)).cuda()
    for call, seed in enumerate((21, 22)):
        rois = synth.crop_rois(seed, 9, 1280, 720, (32, 640), (32, 480))
        ins = [F.as_fkl(frame)] * 9
        want = torch.zeros((9, 3, 64, 128), device="cuda")
        got = torch.full((9, 3, 64, 128), float("nan"), device="cuda")
        _with_workspace(F, p, ins, rois, F.as_fkl(want, F.FKL_LAYOUT_NCHW))
        F.fkl_execute_batch_unfused_static(p.handle, ins, rois, F.as_fkl(got, F.FKL_LAYOUT_NCHW))
        torch.cuda.synchronize()
        assert torch.equal(got.view(torch.int32), want.view(torch.int32)), f"call {call}"
        # and the fused kernel agrees as well
        fused = torch.zeros_like(got)
        F.fkl_execute_batch(p.handle, ins, rois, F.as_fkl(fused, F.FKL_LAYOUT_NCHW))
        torch.cuda.synchronize()
        assert torch.equal(fused.view(torch.int32), got.view(torch.int32))


def test_static_scratch_refuses_oversized_batches(F):
    from paper_2508_07071_gb300 import workloads as W

    # a 3840x2160 NV12 window decodes to 99.5 MB of float32 RGB: over 32 MiB
    p = F.Pipeline(W.nv12_letterbox_chain(F.FKL_BF16))
    frame = torch.zeros((2160 * 3 // 2, 3840), dtype=torch.uint8, device="cuda")
    out = torch.zeros((1, 3, 640, 640), dtype=torch.bfloat16, device="cuda")
    sentinel = out.clone()
    with pytest.raises(F.FklError) as ei:
        F.fkl_execute_batch_unfused_static(p.handle, [F.as_fkl(frame, F.FKL_LAYOUT_NV12)], None,
                                           F.as_fkl(out, F.FKL_LAYOUT_NCHW))
    assert ei.value.status == F.FKL_ERR_INVALID
    assert "static scratch" in str(ei.value)
    torch.cuda.synchronize()
    assert torch.equal(out, sentinel)
