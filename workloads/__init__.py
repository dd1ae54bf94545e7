"""Seeded synthetic inputs shared by the oracle and the GPU path (no method arithmetic)."""
from .circuits import (  # noqa: F401
    Circuit, Op, PATTERN_ORDER, ONE_QUBIT_GATES, ONE_QUBIT_NAMES, SQRT_X, SQRT_Y, SQRT_W,
    fsim, rect_couplers, diag_couplers, make_circuit, grid_circuit, sycamore_like_circuit,
    open_qubits_default, draw_closed_bitstrings, draw_slice_subset, block_base_index,
    open_bit_positions,
)
from .configs import CONFIGS, Workload, workload  # noqa: F401
