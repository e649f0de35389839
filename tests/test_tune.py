"""The schedule autotuner: host logic on the CPU (signature, candidates,
cache), a short tuning run on the GPU."""
import json

import pytest

from paper_1705_05784_gb300 import inputs


def _probs():
    return [inputs.config_2d(48, 1.5, 6.0, 3, (8, 20), 1e4, 8, 6, seed=70 + i, basis=i % 4,
                             restriction=1, alpha=1e-2, krylov=1) for i in range(2)]


def test_signature_keys_the_workload_not_the_field():
    from paper_1705_05784_gb300 import tune
    a, b = _probs(), _probs()
    b[0].perm = b[0].perm * 3.0                      # another field, same kind of problem
    assert tune.signature(a) == tune.signature(b)
    b[1].restriction = 0                             # another option: another workload
    assert tune.signature(a) != tune.signature(b)


def test_candidates_cover_precision_and_restart():
    from paper_1705_05784_gb300 import tune
    c = tune.candidates()
    assert len(c) == len(tune.PRECISION_VARIANTS) * len(tune.RESTARTS)
    assert {x["precision"] for x in c} == {"fp64", "mixed", "mixed_bf16p"}
    q = tune.apply(_probs(), {"precision": "mixed_bf16p", "restart": 20})
    assert all(p.precision == 1 and p.bf16_p == 1 and p.restart == 20 and p.krylov == 1 for p in q)


def test_a_cached_workload_is_not_tuned_again(tmp_path):
    from paper_1705_05784_gb300 import tune
    probs = _probs()
    path = tmp_path / "tune.json"
    want = {"precision": "mixed", "restart": 40}
    path.write_text(json.dumps({tune.signature(probs): {"best": want, "table": []}}))
    best, table = tune.tune(probs, cache=str(path))   # no GPU work: read from the cache
    assert best == want and table == []


@pytest.mark.gpu
def test_tuning_times_every_candidate_and_picks_a_converged_one(tmp_path):
    from paper_1705_05784_gb300 import tune
    probs = _probs()
    cands = [{"precision": "fp64", "restart": 30}, {"precision": "mixed_bf16p", "restart": 20}]
    path = str(tmp_path / "tune.json")
    best, table = tune.tune(probs, cands=cands, cache=path)
    assert len(table) == 2 and all(r["converged"] == r["of"] == 2 for r in table)
    top = max(table, key=lambda r: r["solves_per_s"])
    assert best == {"precision": top["precision"], "restart": top["restart"]}
    assert json.load(open(path))[tune.signature(probs)]["best"] == best
