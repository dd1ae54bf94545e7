"""Global top-k at scale (the paper's k strings of largest p over all
candidates, Sec. III): the GPU selection through the C ABI against the
oracle's lexsort on the same FP64 amplitudes, bit for bit (indices and p),
including heavy ties at the threshold, k = 1, k = all candidates and a
scattered open-bit map."""
import numpy as np
import pytest

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


def _case(G, l, seed, tie_values=None):
    rng = np.random.default_rng(seed)
    if tie_values is None:
        amps = (rng.standard_normal((G, 1 << l)) + 1j * rng.standard_normal((G, 1 << l))) * 2.0 ** -12
    else:
        amps = np.asarray(tie_values)[rng.integers(0, len(tie_values), size=(G, 1 << l))]
    n_bits = l + int(np.ceil(np.log2(max(G, 2)))) + 3
    closed = np.sort(rng.choice(1 << (n_bits - l), size=G, replace=False)).astype(np.int64)
    pos = rng.permutation(n_bits)[:l]  # open qubits at scattered bit positions
    rest = sorted(set(range(n_bits)) - set(pos.tolist()))
    base = np.zeros(G, dtype=np.int64)
    for i, b in enumerate(rest):
        base |= ((closed >> i) & 1) << b
    return amps, base, pos.astype(np.int64)


@pytest.mark.parametrize("G,l,k,inv_f,ties", [
    (256, 16, 1 << 15, 1.0, False),       # 2^24 candidates, the paper's 30-qubit k
    (64, 12, 1, 8.0, False),
    (16, 10, 16 * 1024, 1.0, False),      # k = every candidate
    (128, 12, 5000, 2.0, True),           # many candidates tied at the threshold
    (1, 20, 3000, 1.0, True),
])
def test_global_topk_matches_oracle(E, G, l, k, inv_f, ties):
    import torch
    vals = [0.0, 0.25, -0.25j, 0.5, 0.5j, 0.125 + 0.125j] if ties else None
    amps, base, pos = _case(G, l, seed=G + l + k, tie_values=vals)
    d = torch.as_tensor(amps, device="cuda")
    db = torch.as_tensor(base, device="cuda")
    idx, p = E.topk(d, k, inv_f, db, pos, global_mode=True)
    ri, rp = pp.topk_global(amps, k, inv_f, base, pos)
    assert np.array_equal(idx.cpu().numpy(), ri)
    assert np.array_equal(p.cpu().numpy(), rp)
