"""Tensor-core (tcgen05) GEMM self-test through the C ABI: the stacked-4M real
lowering of a complex GEMM against a plain FP32 CUDA-core GEMM of the same
16-bit inputs (both accumulate in FP32; only the summation order differs).
Every shape runs each tile form (one accumulator per tile, chunked
accumulation, 256-row tiles) into an n-contiguous and an m-contiguous result."""
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [  # (batch, M, N, K) in complex elements
    (1, 128, 64, 32),      # one tile
    (1, 200, 100, 40),     # ragged M, N, K
    (3, 64, 16, 8),        # batched, M < 128, small N
    (2, 256, 128, 64),     # two M tiles, BN = 256
    (1, 130, 4, 4),        # tiny N and K (tile padding), ragged M
    (5, 96, 300, 260),     # several K stages (4-stage ring wraps), ragged N tile
    (1, 1100, 600, 64),    # nine m tiles x five n tiles
    (2, 520, 1030, 100),   # batched, ragged M, N and K across several tiles
    # more tiles than CTAs, so every CTA reuses its accumulator buffers:
    (4, 8192, 256, 256),   # BN = 256, 256-row tiles (both TMEM halves handed back per tile)
    (64, 4096, 16, 16),    # BN = 32: four epilogue tile groups, eight accumulator buffers
    (16, 2000, 32, 36),    # BN = 64, ragged M and K
]


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_18889_gb300 import binding
    return binding


@pytest.mark.parametrize("prec", [1, 2], ids=["bf16", "fp16"])
@pytest.mark.parametrize("shape", SHAPES, ids=[str(s) for s in SHAPES])
def test_tc_gemm_matches_fp32_reference(B, prec, shape):
    err = B.tn_selftest_gemm_tc(*shape, prec=prec, seed=7)
    assert err < 1e-4, err
