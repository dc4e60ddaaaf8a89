"""Host-side checks of the C ABI: the library loads, exports every function
include/fkl.h declares, and validates chains and arguments before touching
the GPU. Nothing here launches a kernel, so it runs without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def F():
    from paper_2508_07071_gb300 import build
    build.build()
    from paper_2508_07071_gb300 import fkl
    return fkl


def declared_functions():
    text = open(os.path.join(ROOT, "include", "fkl.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fkl_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["fkl_pipeline_create", "fkl_execute", "fkl_execute_batch", "fkl_pipeline_destroy",
                 "fkl_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(F):
    lib = ctypes.CDLL(F.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared_functions()) <= set(F.EXPORTS), "binding must cover every declared function"


def test_version(F):
    assert "sm_103a" in F.fkl_version()


def test_struct_layouts_match_header(F):
    assert ctypes.sizeof(F.fkl_tensor) == 8 + 32 + 8 + 4 + 4
    assert ctypes.sizeof(F.fkl_op_desc) == 4 + 32 + 32
    assert ctypes.sizeof(F.fkl_launch_shape) == 16


def _create(F, ops):
    return F.fkl_pipeline_create(ops)


def _status(F, ops):
    try:
        p = F.fkl_pipeline_create(ops)
    except F.FklError as e:
        return e.status
    F.fkl_pipeline_destroy(p)
    return F.FKL_OK


def test_grammar_errors_are_invalid(F):
    # no read first / no write last / read in the middle / unknown op code
    assert _status(F, [F.mul(1.0), F.write_split(F.FKL_F32)]) == F.FKL_ERR_INVALID
    assert _status(F, [F.read_u8c3(), F.resize(4, 4)]) == F.FKL_ERR_INVALID
    assert _status(F, [F.read_u8c3(), F.read_u8c3(), F.write_split(F.FKL_F32)]) == F.FKL_ERR_INVALID
    assert _status(F, [F.read_u8c3(), F._desc(99), F.write_split(F.FKL_F32)]) == F.FKL_ERR_INVALID
    assert _status(F, [F.read_u8c3()]) == F.FKL_ERR_INVALID
    # modifiers after compute ops, bad sizes, bad dtype, bad FP8 scale
    assert _status(F, [F.read_u8c3(), F.mul(1.0), F.resize(4, 4), F.write_split(F.FKL_F32)]) == F.FKL_ERR_INVALID
    assert _status(F, [F.read_u8c3(), F.resize(0, 4), F.write_split(F.FKL_F32)]) == F.FKL_ERR_INVALID
    assert _status(F, [F.read_u8c3(), F.crop(-1, 0, 4, 4), F.write_split(F.FKL_F32)]) == F.FKL_ERR_INVALID
    assert _status(F, [F.read_u8c3(), F.resize(4, 4), F.write_split(77)]) == F.FKL_ERR_INVALID
    assert _status(F, [F.read_nv12(), F.resize(4, 4), F.write_split(F.FKL_E4M3, 0.0)]) == F.FKL_ERR_INVALID
    assert _status(F, [F.read_nv12(), F.resize(4, 4), F.write_split(F.FKL_E4M3)]) == F.FKL_ERR_INVALID


def test_unsupported_chains(F):
    # right grammar, no compiled instantiation
    assert _status(F, [F.read_u8c3(), F.resize(4, 4), F.div(2.0), F.mul(2.0),
                       F.write_split(F.FKL_F32)]) == F.FKL_ERR_UNSUPPORTED
    assert _status(F, [F.read_u8c3(), F.resize(4, 4), F.write_packed(F.FKL_BF16)]) == F.FKL_ERR_UNSUPPORTED
    assert _status(F, [F.read_nv12(), F.resize(4, 4), F.add_sat_u8(3), F.write_split(F.FKL_U8)]) == F.FKL_ERR_UNSUPPORTED
    assert _status(F, [F.read_f32(), F.mul(2.0), F.write_split(F.FKL_F32)]) == F.FKL_ERR_UNSUPPORTED
    # typed chains: MUL, then ADD|SUB, then DIV, each at most once; F32/F64 out
    assert _status(F, [F.read_f32(), F.div(2.0), F.mul(2.0), F.write_packed(F.FKL_F32)]) == F.FKL_ERR_UNSUPPORTED
    assert _status(F, [F.read_u16(), F.mul(2.0), F.mul(2.0), F.write_packed(F.FKL_F32)]) == F.FKL_ERR_UNSUPPORTED
    assert _status(F, [F.read_u16(), F.swap_rb(), F.write_packed(F.FKL_F32)]) == F.FKL_ERR_UNSUPPORTED
    assert _status(F, [F.read_f64(), F.mul(2.0), F.write_split(F.FKL_F16)]) == F.FKL_ERR_UNSUPPORTED
    assert _status(F, [F.read_f64(), F.mul(2.0), F.write_packed(F.FKL_U16)]) == F.FKL_ERR_UNSUPPORTED
    assert _status(F, [F.read_u8c3(), F.resize(4, 4), F.write_split(F.FKL_F64)]) == F.FKL_ERR_UNSUPPORTED
    assert _status(F, [F.read_f64(), F.crop(0, 0, 2, 2), F.write_packed(F.FKL_F64)]) == F.FKL_ERR_INVALID


def test_supported_chains_and_names(F):
    from paper_2508_07071_gb300 import workloads as W
    cases = [
        (W.normalize_chain(224, 224, roi=(320, 200, 640, 480)), "ResizeU8C3>SwapRB>Mul>Sub>Div>WriteSplit<f32>"),
        (W.nv12_letterbox_chain(F.FKL_BF16), "ResizeNV12>Mul>Sub>Div>WriteSplit<bf16>"),
        (W.nv12_letterbox_chain(F.FKL_E4M3), "WriteSplit<e4m3>"),
        (W.vertical_chain([0, 1, 0], [1.0, 2.0, 3.0]), "ReadF32>(Mul|Add)x3>WriteF32"),
        (W.integer_chain(roi=(1, 1, 4, 4), add_k=(1, 2, 3)), "CropU8C3>SwapRB>AddSatU8>WriteU8"),
        ([F.read_u8c3(), F.crop(0, 0, 8, 8), F.mul(2.0), F.write_split(F.FKL_F32)], "ResizeU8C3>Mul"),
        (W.typed_chain(F.FKL_U16, F.FKL_F64, 1 / 255, 0.5, 0.25), "Read<u16>>Cast<f64>>Mul>Sub>Div>Write<f64>"),
        (W.typed_chain(F.FKL_F32, F.FKL_F32, div=3.0), "Read<f32>>Cast<f32>>Div>Write<f32>"),
        (W.typed_chain(F.FKL_F64, F.FKL_F32), "Read<f64>>Cast<f32>>Write<f32>"),
        ([F.read_u8(), F.mul(2.0), F.add(1.0), F.write_packed(F.FKL_F32)], "fused:ReadU8>(Mul|Add)x2"),
        ([F.read_u8(), F.mul(2.0), F.add(1.0), F.write_packed(F.FKL_F64)], "Read<u8>>Cast<f64>>Mul>Sub"),
    ]
    for ops, frag in cases:
        p = F.fkl_pipeline_create(ops)
        try:
            assert frag in F.fkl_pipeline_kernel_name(p)
        finally:
            F.fkl_pipeline_destroy(p)


def test_launch_shapes(F):
    from paper_2508_07071_gb300 import workloads as W
    p = F.fkl_pipeline_create(W.nv12_letterbox_chain(F.FKL_BF16))
    try:
        shapes = F.fkl_pipeline_shapes(p)
        assert len(shapes) > 10
        assert F.fkl_pipeline_get_shape(p) in shapes
        for s in shapes:
            if s[3] <= 0:  # row-staged kernel: tx threads, ty output rows per job, -ry stages
                assert s[0] in (8, 16) and s[1] in (128, 256) and 1 <= s[2] <= 16 and 0 <= -s[3] <= 8
            else:
                assert s[0] in (4, 8, 16) and s[1] * s[2] <= 256 and s[3] in (1, 2)
        assert any(s[3] <= 0 for s in shapes)
        packed = F.fkl_pipeline_create(W.normalize_chain(224, 224, F.FKL_BF16))
        try:  # the packed reader: register shapes and tile-staged shapes (ry = -1, 2 pixels per thread)
            ps = F.fkl_pipeline_shapes(packed)
            assert all(s[3] > 0 or (s[3] == -1 and s[0] <= 4 and s[1] * s[2] <= 256) for s in ps)
            assert any(s[3] == -1 for s in ps)
        finally:
            F.fkl_pipeline_destroy(packed)
        F.fkl_pipeline_set_shape(p, shapes[-1])
        assert F.fkl_pipeline_get_shape(p) == shapes[-1]
        with pytest.raises(F.FklError):
            F.fkl_pipeline_set_shape(p, (3, 16, 8, 1))
        with pytest.raises(F.FklError):
            F.fkl_pipeline_set_shape(p, (8, 32, 32, 1))
    finally:
        F.fkl_pipeline_destroy(p)


def test_execute_validates_before_launch(F):
    """Bad tensors are rejected on the host: no kernel is launched."""
    from paper_2508_07071_gb300 import workloads as W
    p = F.fkl_pipeline_create(W.normalize_chain(16, 8, roi=(0, 0, 32, 16)))
    try:
        src = F._tensor(0x1000, (20, 40, 3), 120, F.FKL_U8, F.FKL_LAYOUT_HWC)
        out = F._tensor(0x2000, (1, 3, 8, 16), 64, F.FKL_F32, F.FKL_LAYOUT_NCHW)
        null_src = F._tensor(0, (20, 40, 3), 120, F.FKL_U8, F.FKL_LAYOUT_HWC)
        bad = {
            "null input": (null_src, out),
            "roi outside": (F._tensor(0x1000, (10, 40, 3), 120, F.FKL_U8, F.FKL_LAYOUT_HWC), out),
            "wrong out dtype": (src, F._tensor(0x2000, (1, 3, 8, 16), 32, F.FKL_F16, F.FKL_LAYOUT_NCHW)),
            "wrong out size": (src, F._tensor(0x2000, (1, 3, 9, 16), 64, F.FKL_F32, F.FKL_LAYOUT_NCHW)),
            "pitch too small": (src, F._tensor(0x2000, (1, 3, 8, 16), 60, F.FKL_F32, F.FKL_LAYOUT_NCHW)),
            "wrong layout": (src, F._tensor(0x2000, (1, 8, 16, 3), 192, F.FKL_F32, F.FKL_LAYOUT_NHWC)),
            "two channels": (F._tensor(0x1000, (20, 40, 2), 80, F.FKL_U8, F.FKL_LAYOUT_HWC), out),
            "input pitch": (F._tensor(0x1000, (20, 40, 3), 100, F.FKL_U8, F.FKL_LAYOUT_HWC), out),
            "input wider than 16384": (F._tensor(0x1000, (20, 16385, 3), 3 * 16385, F.FKL_U8, F.FKL_LAYOUT_HWC),
                                       out),
        }
        for name, (i, o) in bad.items():
            with pytest.raises(F.FklError) as ei:
                F.fkl_execute(p, i, o, stream=0)
            assert ei.value.status == F.FKL_ERR_INVALID, name
        # a resize target beyond 16384 is refused when the pipeline is made
        with pytest.raises(F.FklError) as ei:
            F.fkl_pipeline_create(W.normalize_chain(16385, 8))
        assert ei.value.status == F.FKL_ERR_INVALID
        # batch: per-image ROIs validated too, out must hold n images
        with pytest.raises(F.FklError):
            F.fkl_execute_batch(p, [src, src], [(0, 0, 32, 16), (30, 0, 32, 16)], out, stream=0)
        # vertical chains refuse image tensors; image chains refuse linear ones
        pv = F.fkl_pipeline_create(W.vertical_chain([0], [2.0]))
        try:
            with pytest.raises(F.FklError):
                F.fkl_execute(pv, src, out, stream=0)
            lin = F._tensor(0x3000, (10,), 0, F.FKL_F32, F.FKL_LAYOUT_LINEAR)
            lin2 = F._tensor(0x4000, (11,), 0, F.FKL_F32, F.FKL_LAYOUT_LINEAR)
            with pytest.raises(F.FklError):
                F.fkl_execute(pv, lin, lin2, stream=0)
        finally:
            F.fkl_pipeline_destroy(pv)
    finally:
        F.fkl_pipeline_destroy(p)


def test_nv12_validation(F):
    from paper_2508_07071_gb300 import workloads as W
    p = F.fkl_pipeline_create(W.nv12_letterbox_chain(F.FKL_BF16, out=64))
    try:
        out = F._tensor(0x2000, (1, 3, 64, 64), 128, F.FKL_BF16, F.FKL_LAYOUT_NCHW)
        odd = F._tensor(0x1000, (71, 128), 128, F.FKL_U8, F.FKL_LAYOUT_NV12)
        with pytest.raises(F.FklError):
            F.fkl_execute(p, odd, out, stream=0)
        hwc = F._tensor(0x1000, (72, 128, 3), 384, F.FKL_U8, F.FKL_LAYOUT_HWC)
        with pytest.raises(F.FklError):
            F.fkl_execute(p, hwc, out, stream=0)
    finally:
        F.fkl_pipeline_destroy(p)


def test_unfused_workspace_size_is_the_memory_saved(F):
    """fkl_unfused_workspace_bytes is host arithmetic: two ping-pong float32
    3-channel images, each 256-byte rounded (paper §VI-L memory saving)."""
    from paper_2508_07071_gb300 import workloads as W
    p = F.fkl_pipeline_create(W.normalize_chain(120, 60, roi=(0, 0, 200, 100)))
    try:
        src = F._tensor(0x1000, (100, 200, 3), 600, F.FKL_U8, F.FKL_LAYOUT_HWC)
        out = F._tensor(0x2000, (1, 3, 60, 120), 480, F.FKL_F32, F.FKL_LAYOUT_NCHW)
        n = F.fkl_unfused_workspace_bytes(p, [src], None, out)
        one = (60 * 120 * 12 + 255) // 256 * 256
        assert n == 2 * one
        # one 60x120 float3 image is 86,400 bytes; the paper's 259 KB (§VI-L) is
        # three such intermediates (crop_32F, d_up, d_temp)
        assert 60 * 120 * 12 == 86400 and 3 * 86400 == 259200
    finally:
        F.fkl_pipeline_destroy(p)


def test_device_wait_limit_is_validated_on_the_host(F):
    with pytest.raises(F.FklError) as e:
        F.fkl_set_device_wait_limit(11 * 10**9)
    assert e.value.status == F.FKL_ERR_INVALID
    F.fkl_set_device_wait_limit(5 * 10**8)
    F.fkl_set_device_wait_limit(0)  # back to the default


def test_typed_chain_validation(F):
    """Typed chains check types, lengths and the output size on the host."""
    from paper_2508_07071_gb300 import workloads as W
    p = F.fkl_pipeline_create(W.typed_chain(F.FKL_U16, F.FKL_F64, 2.0, 1.0, 4.0))
    try:
        shapes = F.fkl_pipeline_shapes(p)
        assert shapes and all(s[0] in (8, 16) and s[1] in (128, 256) for s in shapes)
        ok = F._tensor(0x1000, (100,), 0, F.FKL_U16, F.FKL_LAYOUT_LINEAR)
        out2 = F._tensor(0x9000, (200,), 0, F.FKL_F64, F.FKL_LAYOUT_LINEAR)
        bad = {
            "input dtype": ([F._tensor(0x1000, (100,), 0, F.FKL_U8, F.FKL_LAYOUT_LINEAR), ok], out2),
            "lengths differ": ([ok, F._tensor(0x2000, (99,), 0, F.FKL_U16, F.FKL_LAYOUT_LINEAR)], out2),
            "output dtype": ([ok, ok], F._tensor(0x9000, (200,), 0, F.FKL_F32, F.FKL_LAYOUT_LINEAR)),
            "output size": ([ok, ok], F._tensor(0x9000, (199,), 0, F.FKL_F64, F.FKL_LAYOUT_LINEAR)),
            "output layout": ([ok, ok], F._tensor(0x9000, (2, 100, 1, 1), 0, F.FKL_F64, F.FKL_LAYOUT_NCHW)),
            "null input": ([ok, F._tensor(0, (100,), 0, F.FKL_U16, F.FKL_LAYOUT_LINEAR)], out2),
        }
        for name, (ins, o) in bad.items():
            with pytest.raises(F.FklError) as ei:
                F.fkl_execute_batch(p, ins, None, o, stream=0)
            assert ei.value.status == F.FKL_ERR_INVALID, name
        with pytest.raises(F.FklError) as ei:  # typed chains take no ROIs
            F.fkl_execute_batch(p, [ok, ok], [(0, 0, 1, 1), (0, 0, 1, 1)], out2, stream=0)
        assert ei.value.status == F.FKL_ERR_INVALID
        assert F.fkl_unfused_workspace_bytes(p, [ok, ok], None, out2) == 0  # in place on the output
    finally:
        F.fkl_pipeline_destroy(p)


def test_typed_chain_narrow_outputs_parse(F):
    from paper_2508_07071_gb300 import workloads as W
    for dt, name in [(F.FKL_BF16, "bf16"), (F.FKL_F16, "f16")]:
        p = F.fkl_pipeline_create(W.typed_chain(F.FKL_U16, dt, 2.0))
        try:
            assert F.fkl_pipeline_kernel_name(p).endswith(f"Write<{name}>")
        finally:
            F.fkl_pipeline_destroy(p)
    # FP8 needs its scale; packed u8/u16 outputs are not compiled
    assert _status(F, W.typed_chain(F.FKL_F32, F.FKL_E4M3, 2.0)) == F.FKL_ERR_INVALID
    assert _status(F, W.typed_chain(F.FKL_F32, F.FKL_E4M3, 2.0, scale=0.5)) == F.FKL_OK
    assert _status(F, W.typed_chain(F.FKL_F32, F.FKL_U8, 2.0)) == F.FKL_ERR_UNSUPPORTED
    assert _status(F, W.typed_chain(F.FKL_F32, F.FKL_U16, 2.0)) == F.FKL_ERR_UNSUPPORTED
    p = F.fkl_pipeline_create(W.typed_chain(F.FKL_F64, F.FKL_BF16, 2.0))
    try:  # the unfused form keeps one tensor's float32 values in the workspace
        a = F._tensor(0x1000, (1000,), 0, F.FKL_F64, F.FKL_LAYOUT_LINEAR)
        o = F._tensor(0x9000, (3000,), 0, F.FKL_BF16, F.FKL_LAYOUT_LINEAR)
        assert F.fkl_unfused_workspace_bytes(p, [a, a, a], None, o) == 4096
        with pytest.raises(F.FklError) as ei:
            F.fkl_execute_batch_unfused(p, [a, a, a], None, o, 0x100000, 1024, stream=0)
        assert ei.value.status == F.FKL_ERR_INVALID
    finally:
        F.fkl_pipeline_destroy(p)


def test_static_unfused_validates_tensor_chains_before_any_device_call(F):
    from paper_2508_07071_gb300 import workloads as W
    p = F.fkl_pipeline_create(W.typed_chain(F.FKL_F64, F.FKL_BF16, 2.0))
    try:
        a = F._tensor(0x1000, (1000,), 0, F.FKL_F64, F.FKL_LAYOUT_LINEAR)
        short = F._tensor(0x9000, (1999,), 0, F.FKL_BF16, F.FKL_LAYOUT_LINEAR)
        with pytest.raises(F.FklError) as ei:
            F.fkl_execute_batch_unfused_static(p, [a, a], None, short, stream=0)
        assert ei.value.status == F.FKL_ERR_INVALID
    finally:
        F.fkl_pipeline_destroy(p)


def test_static_unfused_refuses_tensors_beyond_its_scratch_before_any_device_call(F):
    """A typed chain writing bf16 keeps one tensor's float32 values in the
    static scratch (32 MiB): 9M elements (36 MB) are refused on the host with
    a message about that scratch, before the scratch's address is looked up."""
    from paper_2508_07071_gb300 import workloads as W
    p = F.fkl_pipeline_create(W.typed_chain(F.FKL_F32, F.FKL_BF16, 2.0))
    try:
        n = 9 * 2**20
        a = F._tensor(0x1000, (n,), 0, F.FKL_F32, F.FKL_LAYOUT_LINEAR)
        o = F._tensor(0x9000, (n,), 0, F.FKL_BF16, F.FKL_LAYOUT_LINEAR)
        with pytest.raises(F.FklError) as ei:
            F.fkl_execute_batch_unfused_static(p, [a], None, o, stream=0)
        assert ei.value.status == F.FKL_ERR_INVALID
        assert "static scratch" in str(ei.value)
        # the caller-workspace form reports what it would need instead
        assert F.fkl_unfused_workspace_bytes(p, [a], None, o) == n * 4
    finally:
        F.fkl_pipeline_destroy(p)


def test_error_messages_are_kept_per_thread_and_truncated(F):
    """fkl_last_error is thread-local text in a fixed buffer (reporting a
    failure allocates nothing); a long message is cut, not overflowed."""
    import threading
    from paper_2508_07071_gb300 import workloads as W
    p = F.fkl_pipeline_create(W.typed_chain(F.FKL_F32, F.FKL_BF16, 2.0))
    try:
        a = F._tensor(0x1000, (10,), 0, F.FKL_F32, F.FKL_LAYOUT_LINEAR)
        o = F._tensor(0x9000, (11,), 0, F.FKL_BF16, F.FKL_LAYOUT_LINEAR)
        with pytest.raises(F.FklError):
            F.fkl_execute_batch(p, [a], None, o, stream=0)
        here = F._lib.fkl_last_error().decode()
        assert "output must hold" in here and len(here) < 512
        seen = []
        t = threading.Thread(target=lambda: seen.append(F._lib.fkl_last_error().decode()))
        t.start()
        t.join()
        assert seen == [""]
        assert F._lib.fkl_last_error().decode() == here
    finally:
        F.fkl_pipeline_destroy(p)


def test_per_op_workspace_and_validation(F):
    """The per-op form sizes two ping-pong sets of chunk intermediates and
    checks its workspace on the host, before any launch."""
    from paper_2508_07071_gb300 import workloads as W
    p = F.fkl_pipeline_create(W.nv12_letterbox_chain(F.FKL_BF16, out=64))
    try:
        src = F._tensor(0x1000, (128, 256), 256, F.FKL_U8, F.FKL_LAYOUT_NV12)
        out = F._tensor(0x2000, (5, 3, 64, 64), 128, F.FKL_BF16, F.FKL_LAYOUT_NCHW)
        slot_in = (256 * 128 * 12 + 767) // 768 * 768   # the decoded source window
        slot = (64 * 64 * 12 + 767) // 768 * 768        # one output-size image
        each = slot_in + slot
        assert F.fkl_per_op_workspace_bytes(p, [src] * 5, None, out, 0) == 5 * each
        assert F.fkl_per_op_workspace_bytes(p, [src] * 5, None, out, 2) == 2 * each
        assert F.fkl_per_op_workspace_bytes(p, [src] * 5, None, out, 999) == 5 * each
        with pytest.raises(F.FklError) as ei:          # workspace too small: refused before any launch
            F.fkl_execute_batch_per_op(p, [src] * 5, None, out, 0x100000, 5 * each - 256, stream=0)
        assert ei.value.status == F.FKL_ERR_INVALID
        with pytest.raises(F.FklError) as ei:          # unaligned workspace
            F.fkl_execute_batch_per_op(p, [src] * 5, None, out, 0x100010, 5 * each, stream=0)
        assert ei.value.status == F.FKL_ERR_INVALID
    finally:
        F.fkl_pipeline_destroy(p)
    pv = F.fkl_pipeline_create(W.vertical_chain([0], [2.0]))
    try:
        lin = F._tensor(0x3000, (10,), 0, F.FKL_F32, F.FKL_LAYOUT_LINEAR)
        with pytest.raises(F.FklError) as ei:
            F.fkl_per_op_workspace_bytes(pv, [lin], None, lin, 0)
        assert ei.value.status == F.FKL_ERR_UNSUPPORTED
    finally:
        F.fkl_pipeline_destroy(pv)
