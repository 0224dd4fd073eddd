"""rms_synth_noalloc: the FP16X3 synthesis entry point that allocates nothing.

It exists for callers that cannot allocate device memory while they process
data (memory reserved up front, or owned by another allocator).  Its results
must match rms_synth's on the same plan and the FP64 oracle, call after call,
although every call reuses the same fixed scratch array (within the FP16X3
tolerance: the two kernels fold their partial sums in different groups), and a
run of calls must leave the device's memory exactly as it found it.  This file
is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import gpu_helpers as gh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rms():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_06250_gb300 as rms
    rms.build()
    rms.load()
    return rms


def _outputs(nlos, nphi):
    dev = torch.device("cuda")
    return (torch.full((nlos, nphi, 2), float("nan"), device=dev),
            torch.full((nlos,), -7, dtype=torch.int32, device=dev),
            torch.zeros(nlos, device=dev), torch.zeros(nlos, device=dev))


@pytest.mark.parametrize("layout", ["chan", "los"])
def test_noalloc_matches_rms_synth(rms, oracle_mod, layout):
    from paper_1810_06250_gb300 import inputs
    cfg = inputs.CONFIGS["lofar"]
    freq, w, phi = inputs.frequencies(cfg), inputs.weights(cfg), inputs.phi_grid(cfg)
    nlos = 20000
    dev = torch.device("cuda")
    with rms.Plan(freq, phi, "fp16x3", weights=w) as plan:
        for call, start in enumerate((0, 50000)):     # two calls in a row, different cubes
            Q, U = inputs.make_cube(cfg, start, nlos)
            if call == 1:
                Q *= 37.5                               # other per-LOS exponents than the first call
                U *= 37.5
            q = torch.from_numpy(inputs.to_layout(Q, layout)).to(dev)
            u = torch.from_numpy(inputs.to_layout(U, layout)).to(dev)
            F0, i0, a0, p0 = _outputs(nlos, cfg.nphi)
            F1, i1, a1, p1 = _outputs(nlos, cfg.nphi)
            rms.rms_synth(plan.handle, q, u, nlos, layout, F0, i0, a0, p0)
            rms.rms_synth_noalloc(plan.handle, q, u, nlos, layout, F1, i1, a1, p1)
            plan.sync()
            Fa, Fb = F0.cpu().numpy(), F1.cpu().numpy()
            per, _ = gh.errors(Fb[..., 0] + 1j * Fb[..., 1], Fa[..., 0] + 1j * Fa[..., 1])
            assert per.max() <= gh.TOL["fp16x3"], per.max()
            # the two kernels fold their FP32 partial sums in different groups, so F may
            # differ in the last bits: each peak map is exact for its own F, and the two
            # agree wherever the top-2 gap of F clears the tolerance
            for F, i, a, p in ((Fa, i0, a0, p0), (Fb, i1, a1, p1)):
                gh.check_peaks_self(F, i.cpu().numpy(), a.cpu().numpy(), p.cpu().numpy(), phi)
            gh.check_peaks_oracle(i1.cpu().numpy(), Fa[..., 0] + 1j * Fa[..., 1], gh.TOL["fp16x3"])
            np.testing.assert_allclose(a1.cpu().numpy(), a0.cpu().numpy(), rtol=2 * gh.TOL["fp16x3"])
            # and against the FP64 oracle on a sample of rows spread over the call
            rows = np.arange(0, nlos, 79)
            op = oracle_mod.plan(freq, "freq", w)
            Fo = oracle_mod.synth(Q[rows], U[rows], op, phi)
            ok, info = gh.gate("fp16x3", Fb[rows][..., 0] + 1j * Fb[rows][..., 1], Fo)
            assert ok, info
            gh.check_peaks_oracle(i1.cpu().numpy()[rows], Fo, gh.TOL["fp16x3"])


def test_noalloc_limits(rms):
    from paper_1810_06250_gb300 import inputs
    cfg = inputs.CONFIGS["tiny"]
    freq, phi = inputs.frequencies(cfg), inputs.phi_grid(cfg)
    q = torch.zeros(cfg.nchan * 8, device="cuda")
    with rms.Plan(freq, phi, "fp16x3") as plan:
        with pytest.raises(rms.RmsError) as e:       # beyond the fixed scratch: rejected, nothing launched
            rms.rms_synth_noalloc(plan.handle, q, q, rms.RMS_NOALLOC_MAX_LOS + 1, "chan", None, q.view(torch.int32))
        assert e.value.status == rms.RMS_ERR_INVALID_ARG
    with rms.Plan(freq, phi, "bf16x3") as plan:
        with pytest.raises(rms.RmsError) as e:
            rms.rms_synth_noalloc(plan.handle, q, q, 8, "chan", None, q.view(torch.int32))
        assert e.value.status == rms.RMS_ERR_UNSUPPORTED


def _device_memory_state(index):
    """(default pool: reserved now, reserved high-water mark, used now, used
    high-water mark; free device bytes) through the CUDA driver API."""
    cu = ctypes.CDLL("libcuda.so.1")
    dev = ctypes.c_int()
    assert cu.cuDeviceGet(ctypes.byref(dev), index) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    vals = []
    for attr in (5, 6, 7, 8):   # CU_MEMPOOL_ATTR_{RESERVED,USED}_MEM_{CURRENT,HIGH} (cuda.h order)
        v = ctypes.c_uint64()
        assert cu.cuMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
        vals.append(v.value)
    free, total = ctypes.c_size_t(), ctypes.c_size_t()
    assert cu.cuMemGetInfo_v2(ctypes.byref(free), ctypes.byref(total)) == 0
    return vals + [free.value], cu, pool


def test_noalloc_allocates_nothing(rms):
    """After the plan exists (which loads the array and the kernels), a run of calls
    changes neither the pool's reserved or used bytes -- not even for a moment:
    the high-water marks are reset first -- nor the device's free memory."""
    from paper_1810_06250_gb300 import inputs
    cfg = inputs.CONFIGS["lofar"]
    freq, w, phi = inputs.frequencies(cfg), inputs.weights(cfg), inputs.phi_grid(cfg)
    nlos = 8192
    dev = torch.device("cuda")
    Q, U = inputs.make_cube(cfg, 0, nlos)
    q = torch.from_numpy(inputs.to_layout(Q, "chan")).to(dev)
    u = torch.from_numpy(inputs.to_layout(U, "chan")).to(dev)
    F, i, a, p = _outputs(nlos, cfg.nphi)
    with rms.Plan(freq, phi, "fp16x3", weights=w) as plan:
        torch.cuda.synchronize()
        before, cu, pool = _device_memory_state(torch.cuda.current_device())
        for attr in (6, 8):         # reset the high-water marks to the current values
            zero = ctypes.c_uint64(0)
            assert cu.cuMemPoolSetAttribute(pool, attr, ctypes.byref(zero)) == 0
        before, _, _ = _device_memory_state(torch.cuda.current_device())
        for _ in range(4):
            rms.rms_synth_noalloc(plan.handle, q, u, nlos, "chan", F, i, a, p)
        plan.sync()
        torch.cuda.synchronize()
        after, _, _ = _device_memory_state(torch.cuda.current_device())
    assert after == before, (before, after)
