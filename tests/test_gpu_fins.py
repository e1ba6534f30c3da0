"""Fin-part comparison (Radon method vs ray-traced optimiser in the non-telecentric
printer) on a 3-fin part: it runs end to end on the GPU and returns valid counts."""
import pytest

pytestmark = pytest.mark.gpu


def test_fins_experiment_three_fins():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2211_03516_gb300 import fins as F
    r = F.fins_experiment(3, iters=10)
    for k in ("ray_traced", "radon"):
        assert 0.0 <= r[k]["ver"] <= 1.0
        assert 0 <= r[k]["fins_formed"] <= 3 and len(r[k]["per_fin"]) == 3
    assert r["ray_traced"]["ver"] < r["radon"]["ver"]
