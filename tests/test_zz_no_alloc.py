"""The allocation-free reference accumulation (GPU).

cg_reference_accumulate_noalloc serves callers that cannot allocate device
memory when they need the reference spectrum (a real-time loop that must not
wait on the allocator, a process whose memory a pool it does not own holds).
It keeps its partial sums in an array compiled into the library.  This test
calls it through the C ABI twice in a row and checks each result against the
allocating entry point cg_reference_accumulate, at the tolerance the
reference test uses (2e-6 relative); a case with more thread blocks' worth of
frames than the array has rows (221 teeth: 148 rows, 10^4 frames) exercises
the grid cap; the first call on a fresh plan leaves the device's free memory
unchanged (the plan did the set-up).  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from tests import workloads as W

torch = pytest.importorskip("torch")
cg = pytest.importorskip("paper_2307_12988_gb300")

pytestmark = pytest.mark.gpu

RTOL = 2e-6


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _noalloc(p, frames, n, dev):
    out = torch.full((p.T,), float("nan"), dtype=torch.float64, device=dev)
    cg._binding.cg_reference_accumulate_noalloc(p.handle, frames, n, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_reference_matches_allocating_entry_point(dev):
    for name in ("paper_rate", "serve4096"):
        w = W.workload(name)
        frames = torch.from_numpy(w["ref_frames"]).to(dev)
        with cg.Plan(*W.plan_args(w)) as p:
            expected = cg.cg_reference_accumulate(p.handle, frames, frames.shape[0])
            for call in range(2):
                got = _noalloc(p, frames, frames.shape[0], dev)
                np.testing.assert_allclose(got, expected, rtol=RTOL, err_msg=f"{name} call {call}")
                np.testing.assert_allclose(got, w["ref"], rtol=RTOL)
            # a smaller second batch right after: results follow the new input
            sub = frames[:17]
            exp_sub = cg.cg_reference_accumulate(p.handle, sub, 17)
            np.testing.assert_allclose(_noalloc(p, sub, 17, dev), exp_sub, rtol=RTOL)


def test_noalloc_more_blocks_than_scratch_rows(dev):
    # 221 teeth leave floor(32768 / 221) = 148 rows of the static array; 10^4
    # frames need far more readout blocks, so the grid is capped at 148
    g = synth.WIDE
    stream = synth.make_stream(g, synth.BASE_SEED + 760)
    rf = synth.frames(stream, 10_000, cavity=False, noise_stream=1, snr_db=30.0)["frames"]
    bins = oracle.tooth_bins(g.sample_rate, g.frame_len, g.tooth_freqs)
    ref = oracle.reference(rf[:500], bins)
    frames = torch.from_numpy(rf).to(dev)
    with cg.Plan(g.sample_rate, g.frame_len, g.tooth_freqs, g.tooth_x, ref) as p:
        assert 32768 // p.T == 148
        assert -(-10_000 // p.info["frames_per_cta"]) > 148
        expected = cg.cg_reference_accumulate(p.handle, frames, 10_000)
        for call in range(2):
            np.testing.assert_allclose(_noalloc(p, frames, 10_000, dev), expected, rtol=RTOL,
                                       err_msg=f"call {call}")
        np.testing.assert_allclose(_noalloc(p, frames[:300], 300, dev), oracle.reference(rf[:300], bins),
                                   rtol=RTOL)


def test_noalloc_first_call_leaves_free_memory_unchanged(dev):
    w = W.workload("tiny")
    frames = torch.from_numpy(w["ref_frames"]).to(dev)
    out = torch.empty(w["geom"].n_teeth, dtype=torch.float64, device=dev)
    with cg.Plan(*W.plan_args(w)) as p:
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        cg._binding.cg_reference_accumulate_noalloc(p.handle, frames, frames.shape[0], out)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    np.testing.assert_allclose(out.cpu().numpy(), w["ref"], rtol=RTOL)


def test_noalloc_rejects_bad_arguments(dev):
    w = W.workload("tiny")
    frames = torch.from_numpy(w["ref_frames"][:4]).to(dev)
    with cg.Plan(*W.plan_args(w)) as p:
        out = torch.empty((p.T,), dtype=torch.float64, device=dev)
        with pytest.raises(cg.CgError):
            cg._binding.cg_reference_accumulate_noalloc(p.handle, frames, 0, out)
        with pytest.raises(cg.CgError):
            cg._binding.cg_reference_accumulate_noalloc(p.handle, frames, 4, None)
        # the binding refuses what the kernel would misuse
        for bad_out in (np.zeros(p.T), out.float(), out[:-1], torch.empty(2 * p.T, dtype=torch.float64,
                                                                            device=dev)[::2]):
            with pytest.raises(cg.CgError, match="CG_ERR_ARG"):
                cg._binding.cg_reference_accumulate_noalloc(p.handle, frames, 4, bad_out)
        with pytest.raises(cg.CgError, match="CG_ERR_ARG"):
            cg._binding.cg_reference_accumulate_noalloc(p.handle, frames, 5, out)
        with pytest.raises(cg.CgError, match="CG_ERR_ARG"):
            cg._binding.cg_reference_accumulate_noalloc(p.handle, frames.float(), 4, out)
        # and the C ABI itself refuses host memory before any launch
        host = np.zeros(p.T)
        lib = cg._binding.load()
        st = lib.cg_reference_accumulate_noalloc(p.handle, frames.data_ptr(), 4,
                                                 host.ctypes.data_as(ctypes.c_void_p), None)
        assert st == cg._binding.CG_ERR_ARG
        host_frames = np.zeros(4 * p.info["frame_len"], dtype=np.int16)
        st = lib.cg_reference_accumulate_noalloc(p.handle, host_frames.ctypes.data_as(ctypes.c_void_p), 4,
                                                 out.data_ptr(), None)
        assert st == cg._binding.CG_ERR_ARG
        cg.cg_check_device(p.handle)
