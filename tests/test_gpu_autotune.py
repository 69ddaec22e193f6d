"""The autotuner's learned cost model (needs a GPU).

The network is trained with the library's own CUDA kernels (forward,
gradient, Adam); its gradients are checked against the float64 CPU oracle
(oracle/mlp_oracle.py).  The gain test measures what the trained model buys
over choosing parameters without it: the thesis's rule (no measurement) and
exhaustive measurement of every candidate."""
import json
import math
import os

import numpy as np
import pytest

import mlp_oracle as mo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def at():
    import torch
    import paper_1503_04955_gb300 as pkg
    from paper_1503_04955_gb300 import autotune
    assert torch.cuda.is_available()
    pkg.buildlib.build()
    return autotune


def test_mlp_kernels_match_oracle(at):
    rng = np.random.default_rng(1)
    model = at.CostModel(seed=3)
    p = model.params.cpu().numpy().astype(np.float64)
    x = rng.normal(0, 1, (300, mo.F)).astype(np.float32)
    t = rng.normal(0, 1, 300).astype(np.float32)
    y = model.predict(x)                      # y_shift is 0 before fit
    assert np.allclose(y, mo.forward(p, x.astype(np.float64)), rtol=1e-4, atol=1e-4)
    loss, g = model.gradient(x, t)
    g_ref = mo.grad(p, x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - mo.loss(p, x, t)) <= 1e-4 * max(1.0, abs(loss))
    assert np.allclose(g, g_ref, rtol=1e-3, atol=1e-5 * np.abs(g_ref).max())
    # one Adam step on the device against the oracle's
    import torch
    lib = at.binding.load()
    pd = torch.tensor(p.astype(np.float32), device="cuda")
    gd = torch.tensor(g_ref.astype(np.float32), device="cuda")
    m1 = torch.zeros_like(pd)
    m2 = torch.zeros_like(pd)
    at.binding._check(lib.dkss_mlp_adam(pd.data_ptr(), gd.data_ptr(), m1.data_ptr(), m2.data_ptr(), 0.01, 1, None),
                      "adam")
    p_ref, _, _ = mo.adam_step(p, g_ref.astype(np.float32).astype(np.float64), 0, 0, 0.01, 1)
    assert np.allclose(pd.cpu().numpy(), p_ref, rtol=1e-5, atol=1e-6)


def test_training_fits_a_smooth_target(at):
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, (400, mo.F)).astype(np.float32)
    t = (3 * x[:, 0] + np.sin(3 * x[:, 1]) + x[:, 2] * x[:, 3]).astype(np.float32)
    model = at.CostModel(seed=5)
    hist = model.fit(x, t, steps=2000, lr=3e-3)
    assert hist[-1] < 0.1 * hist[0]
    assert np.sqrt(np.mean((model.predict(x) - t) ** 2)) < 0.15


TRAIN = [1 << 12, 3 << 12, 1 << 14, 3 << 14, 1 << 16, 3 << 16, 1 << 18, 3 << 18, 1 << 20, 3 << 20, 1 << 22]
HELD_OUT = [1 << 13, 3 << 13, 1 << 15, 1 << 17, 3 << 17, 1 << 19, 1 << 21]


def test_cost_model_gain_over_rule_and_exhaustive_search(at):
    train = at.collect(TRAIN)
    held = at.collect(HELD_OUT)
    model = at.CostModel(seed=7)
    model.fit(np.stack([r[0] for r in train]), np.array([r[1] for r in train]), steps=4000, lr=3e-3)
    report = []
    tot = {"best": 0.0, "rule": 0.0, "model1": 0.0, "model3": 0.0}
    trials = {"exhaustive": 0, "model3": 0}
    for n in HELD_OUT:
        rows = [r for r in held if r[4] == n]
        ms = {json.dumps(r[2], sort_keys=True): r[3] for r in rows}
        cands = [r[2] for r in rows]
        best = min(r[3] for r in rows)
        rule = ms[json.dumps(at.rule_choice(n, cands), sort_keys=True)]
        pred = model.predict(np.stack([r[0] for r in rows]))
        order = np.argsort(pred)
        m1 = rows[order[0]][3]
        m3 = min(rows[i][3] for i in order[:3])
        tot["best"] += best
        tot["rule"] += rule
        tot["model1"] += m1
        tot["model3"] += m3
        trials["exhaustive"] += len(rows)
        trials["model3"] += 3
        report.append({"n_bits": n, "candidates": len(rows), "best_ms": round(best, 4), "rule_ms": round(rule, 4),
                       "model_top1_ms": round(m1, 4), "model_top3_ms": round(m3, 4)})
    out = os.environ.get("DKSS_AUTOTUNE_REPORT")
    if out:
        with open(out, "w") as f:
            json.dump({"held_out": report, "totals_ms": tot, "trials": trials}, f, indent=1)
    print(json.dumps({"totals_ms": tot, "trials": trials}))
    # the model's 3 measured candidates beat the rule and come close to measuring all of them
    assert tot["model3"] <= tot["rule"]
    assert tot["model3"] <= 1.15 * tot["best"]
    assert trials["model3"] < trials["exhaustive"] / 4
