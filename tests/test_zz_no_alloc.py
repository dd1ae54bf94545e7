"""tn_contract_slices_noalloc: the contraction for callers that cannot allocate
device memory (their device memory belongs to another allocator, or their loop
may not allocate).  It uses the library's static 64 MiB device workspace
instead of a caller-allocated one; its output must match tn_contract_slices
on the same plan and slices, on two calls in a row (the array keeps the
previous call's contents)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

C64_TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_18889_gb300 import binding as B
    from paper_2406_18889_gb300 import engine as E
    return torch, B, E


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_workspace_entry_point_twice(env):
    torch, B, E = env
    w = W.workload("grid3x4_d8", cycles=10, l=6, G=8)
    prep = E.prepare(w, n_sliced=4)
    plan = E.Plan(prep.tn, prep.tree, max_slice_batch=8)
    assert plan.info["workspace_bytes"] <= (64 << 20)
    stream = torch.cuda.current_stream().cuda_stream
    ids = np.array([3, 0, 7, 12, 5, 9, 15, 1, 2, 11, 6], dtype=np.int64)  # ragged: 8 + 3
    ref = plan.contract(ids).cpu().numpy()
    for _ in range(2):
        out = torch.full((plan.G, plan.J), float("nan"), dtype=torch.complex128, device="cuda")
        B.tn_contract_slices_noalloc(plan.handle, ids, out.data_ptr(), 0, stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert _rel(got, ref) <= C64_TOL
    # accumulate = 1 adds to the previous contents
    B.tn_contract_slices_noalloc(plan.handle, ids, out.data_ptr(), 1, stream)
    torch.cuda.synchronize()
    assert _rel(out.cpu().numpy(), 2 * ref) <= C64_TOL
    plan.close()


def test_noalloc_calls_allocate_no_device_memory(env):
    # the defining property: after a first call (which loads the kernels and
    # looks up the static array's address), further calls leave the device's
    # free memory, as the driver reports it, unchanged
    torch, B, E = env
    w = W.workload("grid3x4_d8", cycles=10, l=6, G=8)
    prep = E.prepare(w, n_sliced=4)
    plan = E.Plan(prep.tn, prep.tree, max_slice_batch=8, own_workspace=False)
    stream = torch.cuda.current_stream().cuda_stream
    ids = np.arange(16, dtype=np.int64)
    out = torch.zeros((plan.G, plan.J), dtype=torch.complex128, device="cuda")
    B.tn_contract_slices_noalloc(plan.handle, ids, out.data_ptr(), 0, stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for acc in (0, 1, 1, 0):
        B.tn_contract_slices_noalloc(plan.handle, ids, out.data_ptr(), acc, stream)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    plan.close()


def test_noalloc_rejects_plan_beyond_static_workspace(env):
    torch, B, E = env
    w = W.workload("grid4x6_d14")
    prep = E.prepare(w)
    rank, edges, data = E.flatten_network(prep.tn)
    h = B.tn_plan_create(rank, edges, prep.tn.edge_dim, data, prep.tn.open_edges, prep.tn.block_edge,
                         np.asarray(prep.tree.pairs).reshape(-1), prep.tree.sliced_edges,
                         max_slice_batch=64, stream=torch.cuda.current_stream().cuda_stream)
    assert B.tn_plan_query(h)["workspace_bytes"] > (64 << 20)
    out = torch.zeros((64, 1024), dtype=torch.complex128, device="cuda")
    with pytest.raises(B.TNError) as ei:
        B.tn_contract_slices_noalloc(h, np.arange(64), out.data_ptr(), 0,
                                     torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == 1 and "static workspace" in str(ei.value)
    assert torch.count_nonzero(out).item() == 0
    B.tn_plan_destroy(h)
