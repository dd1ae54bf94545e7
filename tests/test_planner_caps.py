"""Memory cap vs time complexity of the planner (paper Sec. III: slicing trades
memory for repeated work).  For a fixed path the greedy slicer's choices do not
depend on the cap, only where it stops, and slicing one more bond multiplies
every step's cost by 1 or 2; so the best total found can only fall as the cap
rises, and every tree found respects its cap."""
import pytest

import workloads as W
from paper_2406_18889_gb300 import network as N
from paper_2406_18889_gb300 import pathfind as P


@pytest.mark.parametrize("method", ["partition", "greedy"])
def test_memory_cap_sweep_monotone(method):
    w = W.workload("grid4x6_d14")
    tn = N.circuit_network(w.circuit, w.open_qubits, w.closed_qubits, w.closed_bits)
    caps = [12, 14, 16, 18, 20, 24, 40]
    res = P.memory_cap_sweep(tn, caps, method=method)
    assert [r["cap_log2"] for r in res] == caps
    found = [r for r in res if "total" in r]
    assert len(found) >= 5
    for r in found:
        assert r["log2_max_intermediate"] <= r["cap_log2"] + 1e-9
        assert r["total"] == pytest.approx(r["cost_per_slice"] * 2.0 ** r["n_sliced"], rel=1e-12)
    for a, b in zip(found, found[1:]):
        assert b["total"] <= a["total"] * (1 + 1e-12)
        assert b["n_sliced"] <= a["n_sliced"] or b["path"] != a["path"]
    # a cap above every intermediate needs no slicing at all
    assert found[-1]["n_sliced"] == 0
