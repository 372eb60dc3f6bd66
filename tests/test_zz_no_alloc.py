"""The allocation-free reference accumulation (GPU).

cg_reference_accumulate_noalloc serves callers that cannot allocate device
memory when they need the reference spectrum (a real-time loop that must not
wait on the allocator, a process whose memory a pool it does not own holds).
It keeps its partial sums in an array compiled into the library.  This test
calls it through the C ABI twice in a row and checks each result against the
allocating entry point cg_reference_accumulate, at the tolerance the
reference test uses (2e-6 relative).  The file is named to be collected last.
"""
import numpy as np
import pytest

from tests import workloads as W

torch = pytest.importorskip("torch")
cg = pytest.importorskip("paper_2307_12988_gb300")

pytestmark = pytest.mark.gpu

RTOL = 2e-6


def test_noalloc_reference_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    for name in ("paper_rate", "serve4096"):
        w = W.workload(name)
        frames = torch.from_numpy(w["ref_frames"]).to(dev)
        with cg.Plan(*W.plan_args(w)) as p:
            expected = cg.cg_reference_accumulate(p.handle, frames, frames.shape[0])
            for call in range(2):
                out = torch.full((p.T,), float("nan"), dtype=torch.float64, device=dev)
                cg._binding.cg_reference_accumulate_noalloc(p.handle, frames, frames.shape[0], out)
                torch.cuda.synchronize()
                got = out.cpu().numpy()
                np.testing.assert_allclose(got, expected, rtol=RTOL, err_msg=f"{name} call {call}")
                np.testing.assert_allclose(got, w["ref"], rtol=RTOL)
            # a smaller second batch right after: results follow the new input
            sub = frames[:17]
            exp_sub = cg.cg_reference_accumulate(p.handle, sub, 17)
            out = torch.empty((p.T,), dtype=torch.float64, device=dev)
            cg._binding.cg_reference_accumulate_noalloc(p.handle, sub, 17, out)
            torch.cuda.synchronize()
            np.testing.assert_allclose(out.cpu().numpy(), exp_sub, rtol=RTOL)


def test_noalloc_rejects_bad_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = W.workload("tiny")
    dev = torch.device("cuda:0")
    frames = torch.from_numpy(w["ref_frames"][:4]).to(dev)
    with cg.Plan(*W.plan_args(w)) as p:
        out = torch.empty((p.T,), dtype=torch.float64, device=dev)
        with pytest.raises(cg.CgError):
            cg._binding.cg_reference_accumulate_noalloc(p.handle, frames, 0, out)
        with pytest.raises(cg.CgError):
            cg._binding.cg_reference_accumulate_noalloc(p.handle, frames, 4, None)
