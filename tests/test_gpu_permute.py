"""tn_permute (bit-permutation transpose) against NumPy's transpose of the same
2^r tensor viewed with 2-wide axes."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_18889_gb300 import binding
    return binding


def _reference(x, out_bit):
    r = len(out_bit)
    # axis a of the (2,)*r view holds bit r-1-a; output bit out_bit[i] takes input bit i
    t = x.reshape((2,) * r)
    src_axis_of_out_axis = [None] * r
    for i, o in enumerate(out_bit):
        src_axis_of_out_axis[r - 1 - o] = r - 1 - i
    return np.ascontiguousarray(t.transpose(src_axis_of_out_axis)).reshape(-1)


@pytest.mark.parametrize("r,seed", [(3, 0), (10, 1), (14, 2), (20, 3)])
@pytest.mark.parametrize("elem", [4, 8])
def test_permute_matches_numpy(B, r, seed, elem):
    import torch
    rng = np.random.default_rng(seed)
    out_bit = rng.permutation(r).astype(np.int32)
    dtype = np.uint32 if elem == 4 else np.uint64
    x = rng.integers(0, 2 ** 31, size=1 << r).astype(dtype)
    tdt = torch.int32 if elem == 4 else torch.int64
    din = torch.as_tensor(x.view(np.int32 if elem == 4 else np.int64), device="cuda")
    dout = torch.empty_like(din)
    B.tn_permute(din.data_ptr(), dout.data_ptr(), out_bit, elem, torch.cuda.current_stream().cuda_stream)
    got = dout.cpu().numpy().view(dtype)
    assert np.array_equal(got, _reference(x, out_bit))
    assert tdt is not None


def test_permute_rejects_non_permutation(B):
    import torch
    d = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(B.TNError):
        B.tn_permute(d.data_ptr(), d.data_ptr() + 128, [0, 1, 1, 3], 8)
