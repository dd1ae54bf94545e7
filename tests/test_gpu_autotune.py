"""Per-step launch-form tuning of the tensor-core steps (tn_plan_autotune): the
chosen forms are valid, the results do not change, and forms round-trip
through the engine's cache."""
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


def test_autotune_keeps_results_and_round_trips(E, tmp_path):
    from paper_2406_18889_gb300 import binding as B
    w = W.workload("grid4x6_d14")
    prep = E.prepare(w)
    flags = B.TN_FLAG_HOIST_INVARIANT
    plan = E.Plan(prep.tn, prep.tree, prec="fp16", flags=flags, max_slice_batch=64)
    before = plan.contract().cpu().numpy()
    k = plan.steps()["kinds"]
    tuned = ((k & 8) > 0) & ((k & 4) == 0)
    cache = str(tmp_path / "forms.json")
    forms = plan.autotune(reps=1, cache=cache)
    assert forms.shape == (len(k), 2)
    assert (forms[tuned][:, 0] > 0).all() and (forms[~tuned] == 0).all()
    assert set(forms[tuned][:, 1]) <= {1, 2}
    after = plan.contract().cpu().numpy()
    # every form runs each output's MMAs over K in the same order
    assert pp.relative_l2(after, before) <= 1e-6
    # a second plan of the same workload takes the cached forms without timing
    plan2 = E.Plan(prep.tn, prep.tree, prec="fp16", flags=flags, max_slice_batch=64)
    forms2 = plan2.autotune(cache=cache)
    assert np.array_equal(forms2, forms)
    assert pp.relative_l2(plan2.contract().cpu().numpy(), before) <= 1e-6
    plan.close()
    plan2.close()


def test_complex64_plan_has_nothing_to_tune(E):
    w = W.workload("grid3x4_d8", cycles=10, l=6, G=8)
    prep = E.prepare(w, n_sliced=3, restarts=1)
    plan = E.Plan(prep.tn, prep.tree, prec="c64", max_slice_batch=8)
    forms = plan.autotune(reps=1)
    assert (forms == 0).all()
    plan.close()
