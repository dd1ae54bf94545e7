"""The slices of one problem split over ranks (multirank.py), on one GPU: each
"rank" contracts its share of the slice ids into an FP64 partial, the partials
are summed in rank order by tn_sum_partials, and the result is compared with
the single-rank sum and with the oracle; top-k of the reduced amplitudes is
the same as the single-rank one.  (Ranks run one after another in one process:
they share no kernels that wait on one another.)"""
import numpy as np
import pytest

import workloads as W
from oracle import einsum_tn as et
from oracle import postprocess as pp
from parity_checks import assert_amplitudes_close

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


def test_sum_partials_is_the_rank_ordered_fp64_sum(E):
    import torch
    from paper_2406_18889_gb300 import binding as B
    rng = np.random.default_rng(7)
    parts = rng.standard_normal((5, 3, 1000)) + 1j * rng.standard_normal((5, 3, 1000))
    parts[2] *= 1e-12  # magnitudes far apart: the order of the additions shows in the bits
    ref = parts[0].copy()
    for p in parts[1:]:
        ref = ref + p
    d_parts = torch.as_tensor(parts, device="cuda")
    out = torch.full((3, 1000), 7.0 + 0j, dtype=torch.complex128, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    B.tn_sum_partials(d_parts.data_ptr(), 5, 3000, out.data_ptr(), 0, s)
    assert np.array_equal(out.cpu().numpy(), ref)
    B.tn_sum_partials(d_parts.data_ptr(), 5, 3000, out.data_ptr(), 1, s)  # adds to the previous sum
    acc = ref.copy()
    for p in parts:
        acc = acc + p
    assert np.array_equal(out.cpu().numpy(), acc)
    B.tn_sum_partials(d_parts.data_ptr(), 0, 3000, out.data_ptr(), 0, s)  # no parts: zeros
    assert torch.count_nonzero(out).item() == 0
    with pytest.raises(B.TNError):
        B.tn_sum_partials(d_parts.data_ptr(), -1, 3000, out.data_ptr(), 0, s)


@pytest.mark.parametrize("world", [2, 3, 8])
def test_slices_split_over_ranks_on_one_gpu(E, world):
    import torch
    from paper_2406_18889_gb300 import binding as B
    from paper_2406_18889_gb300 import multirank as MR
    w = W.workload("grid3x4_d8", cycles=10, l=6, G=8)
    bonds = [(q, 1) for q in range(5)]
    prep = E.prepare(w, sliced_wires=bonds)
    ids = W.draw_slice_subset(32, 13, seed=3)
    plan = E.Plan(prep.tn, prep.tree, max_slice_batch=4)
    single = plan.contract(ids).cpu().numpy()
    parts = torch.stack([plan.contract(MR.partition(ids, r, world)) for r in range(world)])
    out = torch.empty_like(parts[0])
    B.tn_sum_partials(parts.data_ptr(), world, out.numel(), out.data_ptr(), 0,
                      torch.cuda.current_stream().cuda_stream)
    got = out.cpu().numpy()
    assert pp.relative_l2(got, single) <= 1e-12  # FP64 sums of the same complex64 slices
    net = et.build_network(w.circuit, w.open_qubits, w.closed_qubits, w.closed_bits)
    assert_amplitudes_close(got, et.contract(net, bonds, ids), 1e-5)
    base = torch.as_tensor(w.block_base(), device="cuda")
    i1, p1 = E.topk(out, 8, 32 / 13, base, w.open_bit_pos())
    i0, p0 = E.topk(torch.as_tensor(single, device="cuda"), 8, 32 / 13, base, w.open_bit_pos())
    assert np.array_equal(i1.cpu().numpy(), i0.cpu().numpy())
    # the one-process form of contract_partitioned: no collective, the plan's own sum
    one = MR.contract_partitioned(plan, ids, None, 1, 0)
    assert np.array_equal(one.cpu().numpy(), single)
    plan.close()
