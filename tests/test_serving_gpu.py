"""The serving loop (fkl_server_*): continuous batching of requests of mixed
image sizes, admission by free device memory, persistent kernel with a device
queue; every result must be the same alone as in the mix."""
import time

import numpy as np
import pytest

import oracle as O
from paper_2508_07071_gb300 import synth
from parity import check_output, copy_device

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OUT = 224


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2508_07071_gb300 import build
    build.build()
    from paper_2508_07071_gb300 import fkl
    return fkl


@pytest.fixture(scope="module")
def pool():
    """Pinned host images of mixed sizes (requests pick from this pool)."""
    rng = np.random.default_rng(41)
    imgs = []
    for k in range(24):
        w, h = int(rng.integers(320, 1281)), int(rng.integers(240, 721))
        imgs.append(torch.from_numpy(synth.packed_image(100 + k, h, w)).pin_memory())
    return imgs


def make_requests(pool, n_req, seed, max_images=8):
    rng = np.random.default_rng(seed)
    return [list(rng.integers(0, len(pool), int(rng.integers(1, max_images + 1)))) for _ in range(n_req)]


def pipeline(F):
    from paper_2508_07071_gb300 import workloads as W
    return F.Pipeline(W.normalize_chain(OUT, OUT, out_dtype=F.FKL_F16))


def result(F, out):
    n = out.dims[0]
    nbytes = n * 3 * OUT * out.pitch_bytes
    raw = copy_device(out.data, nbytes)
    return raw.view(torch.float16).view(n, 3, OUT, out.pitch_bytes // 2)[..., :OUT].clone()


def serve(F, srv, pool, requests, concurrent=True):
    outs = []
    if concurrent:
        ids = [F.fkl_server_submit(srv, [F.as_fkl(pool[i]) for i in req]) for req in requests]
        for rid in ids:
            outs.append(result(F, F.fkl_server_wait(srv, rid, 30000)))
            F.fkl_server_release(srv, rid)
    else:
        for req in requests:
            rid = F.fkl_server_submit(srv, [F.as_fkl(pool[i]) for i in req])
            outs.append(result(F, F.fkl_server_wait(srv, rid, 30000)))
            F.fkl_server_release(srv, rid)
    return outs


def test_results_same_alone_and_in_the_mix_and_match_oracle(F, pool):
    from paper_2508_07071_gb300 import workloads as W
    p = pipeline(F)
    srv = F.fkl_server_create(p.handle, F.FKL_SERVE_PERSISTENT, max_inflight=16, arena_bytes=1 << 30)
    try:
        reqs = make_requests(pool, 20, 1)
        mixed = serve(F, srv, pool, reqs, concurrent=True)
        alone = serve(F, srv, pool, reqs[:6], concurrent=False)
        for a, b in zip(alone, mixed[:6]):
            assert torch.equal(a.view(torch.int16), b.view(torch.int16))
        for r, out in list(zip(reqs, mixed))[:3]:
            for j, idx in enumerate(r[:2]):
                src = pool[idx].numpy()
                want = O.preprocess_packed(src, (0, 0, src.shape[1], src.shape[0]), OUT, OUT, swap=True,
                                           mul=1 / 255, sub=W.IMAGENET_MEAN, div=W.IMAGENET_STD)
                check_output(out[j], want, "f16", 1.0, "served image")
        st = F.fkl_server_get_stats(srv)
        assert st.completed == 26 and st.images_completed == sum(map(len, reqs)) + sum(map(len, reqs[:6]))
    finally:
        F.fkl_server_destroy(srv)


def test_modes_agree_bitwise(F, pool):
    p = pipeline(F)
    reqs = make_requests(pool, 8, 2)
    results = {}
    for mode in (F.FKL_SERVE_PERSISTENT, F.FKL_SERVE_BATCH, F.FKL_SERVE_UNFUSED):
        srv = F.fkl_server_create(p.handle, mode, max_inflight=8, arena_bytes=1 << 30)
        try:
            results[mode] = serve(F, srv, pool, reqs)
        finally:
            F.fkl_server_destroy(srv)
    for a, b, c in zip(*results.values()):
        assert torch.equal(a.view(torch.int16), b.view(torch.int16))
        assert torch.equal(a.view(torch.int16), c.view(torch.int16))


def test_admission_by_device_memory(F, pool):
    p = pipeline(F)
    big = [i for i in range(len(pool)) if pool[i].shape[0] * pool[i].shape[1] > 500_000][:3]
    one = sum(pool[i].numel() for i in big) + 3 * 3 * OUT * OUT * 2
    srv = F.fkl_server_create(p.handle, F.FKL_SERVE_PERSISTENT, max_inflight=16,
                              arena_bytes=int(one * 2.5) + (1 << 20))
    try:
        ids = [F.fkl_server_submit(srv, [F.as_fkl(pool[i]) for i in big]) for _ in range(6)]
        st = F.fkl_server_get_stats(srv)
        assert st.submitted == 6
        outs = []
        for rid in ids:
            outs.append(result(F, F.fkl_server_wait(srv, rid, 30000)))
            F.fkl_server_release(srv, rid)
        for o in outs[1:]:
            assert torch.equal(o.view(torch.int16), outs[0].view(torch.int16))
        st = F.fkl_server_get_stats(srv)
        assert st.completed == 6 and st.arena_peak_bytes <= int(one * 2.5) + (1 << 20)
        with pytest.raises(F.FklError):  # could never fit (even as staged tap rows: 24 images)
            F.fkl_server_submit(srv, [F.as_fkl(pool[i]) for i in big] * 8)
    finally:
        F.fkl_server_destroy(srv)


def test_idle_kernel_exits_and_is_relaunched(F, pool):
    p = pipeline(F)
    srv = F.fkl_server_create(p.handle, F.FKL_SERVE_PERSISTENT, max_inflight=4, arena_bytes=1 << 28,
                              idle_us=2000)
    try:
        first = serve(F, srv, pool, [[0, 1]])
        time.sleep(0.05)                    # well past the 2 ms idle timeout
        second = serve(F, srv, pool, [[0, 1]])
        assert torch.equal(first[0].view(torch.int16), second[0].view(torch.int16))
        assert F.fkl_server_get_stats(srv).kernel_launches >= 2
        info_ok = True
    finally:
        F.fkl_server_destroy(srv)
    assert info_ok


def test_request_times_and_destroy_with_work_in_flight(F, pool):
    p = pipeline(F)
    srv = F.fkl_server_create(p.handle, F.FKL_SERVE_PERSISTENT, max_inflight=8, arena_bytes=1 << 30)
    rid = F.fkl_server_submit(srv, [F.as_fkl(pool[i]) for i in range(8)])
    F.fkl_server_wait(srv, rid, 30000)
    info = F.fkl_server_request_info(srv, rid)
    assert info.state == 3 and info.n_images == 8
    assert info.t_submit <= info.t_admit <= info.t_ready <= info.t_done
    for _ in range(5):                      # left in flight on purpose
        F.fkl_server_submit(srv, [F.as_fkl(pool[i]) for i in range(4)])
    t0 = time.time()
    F.fkl_server_destroy(srv)
    assert time.time() - t0 < 15.0


def test_largest_and_smallest_images_match_oracle(F):
    """The config's extremes (3840x2160, 320x240 and the two mixed shapes),
    in one request and in a mix with others, element by element against the
    oracle: the resize factors and the 64-bit row offsets of a 4K frame."""
    from paper_2508_07071_gb300 import workloads as W
    sizes = [(2160, 3840), (240, 320), (240, 3840), (2160, 320), (721, 1283)]
    imgs = [torch.from_numpy(synth.packed_image(500 + k, h, w)).pin_memory() for k, (h, w) in enumerate(sizes)]
    p = pipeline(F)
    for mode in (F.FKL_SERVE_PERSISTENT, F.FKL_SERVE_UNFUSED):
        srv = F.fkl_server_create(p.handle, mode, max_inflight=8, arena_bytes=1 << 30)
        try:
            reqs = [[0, 1, 2, 3, 4], [4, 3], [0], [1, 0]]
            outs = serve(F, srv, imgs, reqs)
        finally:
            F.fkl_server_destroy(srv)
        want = []
        for im in imgs:
            src = im.numpy()
            want.append(O.preprocess_packed(src, (0, 0, src.shape[1], src.shape[0]), OUT, OUT, swap=True,
                                            mul=1 / 255, sub=W.IMAGENET_MEAN, div=W.IMAGENET_STD))
        for r, out in zip(reqs, outs):
            for j, idx in enumerate(r):
                check_output(out[j], want[idx], "f16", 1.0, f"mode {mode} image {sizes[idx]}")


def test_requests_overlap_on_the_device(F, pool):
    """Continuous batching: requests submitted together are admitted and
    published while earlier ones are still running, so some later request's
    work is on the device (published to the kernel's queue) before an earlier
    request has finished."""
    p = pipeline(F)
    srv = F.fkl_server_create(p.handle, F.FKL_SERVE_PERSISTENT, max_inflight=16, arena_bytes=1 << 30)
    try:
        reqs = make_requests(pool, 12, 7, max_images=6)
        ids = [F.fkl_server_submit(srv, [F.as_fkl(pool[i]) for i in r]) for r in reqs]
        infos = []
        for rid in ids:
            F.fkl_server_wait(srv, rid, 30000)
            infos.append(F.fkl_server_request_info(srv, rid))
            F.fkl_server_release(srv, rid)
    finally:
        F.fkl_server_destroy(srv)
    overlapped = [(i, j) for i in range(len(infos)) for j in range(i + 1, len(infos))
                  if infos[j].t_ready < infos[i].t_done and infos[j].t_admit < infos[i].t_done]
    assert overlapped, [(x.t_admit, x.t_ready, x.t_done) for x in infos]
    # FIFO admission: no request is admitted before one submitted earlier
    assert all(infos[k].t_admit <= infos[k + 1].t_admit for k in range(len(infos) - 1))


def test_persistent_mode_refuses_pageable_images(F, pool):
    """The persistent kernel reads the host images itself: pageable memory is
    refused at submit, pinned memory accepted."""
    p = pipeline(F)
    srv = F.fkl_server_create(p.handle, F.FKL_SERVE_PERSISTENT, max_inflight=4, arena_bytes=1 << 28)
    try:
        pageable = torch.from_numpy(synth.packed_image(7, 300, 400))
        with pytest.raises(F.FklError) as ei:
            F.fkl_server_submit(srv, [F.as_fkl(pageable)])
        assert ei.value.status == F.FKL_ERR_INVALID
        rid = F.fkl_server_submit(srv, [F.as_fkl(pool[0])])
        F.fkl_server_wait(srv, rid, 30000)
        F.fkl_server_release(srv, rid)
    finally:
        F.fkl_server_destroy(srv)
