"""Failure detection without faulting the GPU: a bounded device wait that runs
out reports TN_ERR_TIMEOUT and leaves the context usable; injected host-side
failures reject calls before any device work; an interrupted checkpointed
contraction resumes to the same bits."""
import numpy as np
import pytest

import workloads as W
from oracle import postprocess as pp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_18889_gb300 import engine
    return engine


def test_bounded_wait_times_out_and_context_survives(E):
    import torch
    from paper_2406_18889_gb300 import binding as B
    with pytest.raises(B.TNError) as ei:
        B.tn_selftest_bounded_wait(2_000_000)  # 2 ms on a barrier nothing completes
    assert ei.value.status == B.TN_ERR_TIMEOUT
    # the context still runs work afterwards
    w = W.workload("grid3x4_d8", l=6, G=8)
    prep = E.prepare(w, n_sliced=2)
    plan = E.Plan(prep.tn, prep.tree, max_slice_batch=4)
    a = plan.contract().cpu().numpy()
    assert np.isfinite(a).all() and np.abs(a).max() > 0
    torch.cuda.synchronize()


def test_fp32_peak_is_plausible(E):
    from paper_2406_18889_gb300 import binding as B
    t = B.tn_selftest_fp32_peak()
    assert 10.0 < t < 200.0, t  # GB300: 152 SMs x 128 FP32 lanes x 2 flop x ~2 GHz ~ 80 TFLOP/s


def test_injected_stream_fault_leaves_output_untouched(E, monkeypatch):
    import torch
    from paper_2406_18889_gb300 import binding as B
    w = W.workload("grid3x4_d8", l=6, G=8)
    prep = E.prepare(w, n_sliced=2)
    plan = E.Plan(prep.tn, prep.tree, max_slice_batch=4)
    out = torch.full((8, 64), 3.0, dtype=torch.complex128, device="cuda")
    monkeypatch.setenv("TN_FAULT", "stream")
    with pytest.raises(B.TNError) as ei:
        plan.contract(out=out)
    assert ei.value.status == B.TN_ERR_CUDA
    assert torch.all(out == 3.0).item()
    monkeypatch.delenv("TN_FAULT")
    plan.contract(out=out)
    assert not torch.all(out == 3.0).item()


class _Stop(Exception):
    pass


def test_checkpoint_resume_is_bit_identical(E, tmp_path):
    w = W.workload("grid3x4_d8", cycles=10, l=6, G=8)
    prep = E.prepare(w, n_sliced=5)
    plan = E.Plan(prep.tn, prep.tree, max_slice_batch=4)
    ids = W.draw_slice_subset(32, 20, seed=3)
    whole = E.contract_checkpointed(plan, ids, str(tmp_path / "a.npz"), chunk=4).cpu().numpy()

    def stop_after_two(i, done):
        if i == 1:
            raise _Stop()

    path = str(tmp_path / "b.npz")
    with pytest.raises(_Stop):
        E.contract_checkpointed(plan, ids, path, chunk=4, on_chunk=stop_after_two)
    ck = np.load(path)
    assert int(ck["done"]) == 8
    resumed = E.contract_checkpointed(plan, ids, path, chunk=4).cpu().numpy()
    assert np.array_equal(whole, resumed)
    assert pp.relative_l2(resumed, plan.contract(ids).cpu().numpy()) <= 1e-12
