"""Host logic of the fin-part comparison: the per-fin formation count on doses built by
hand (no GPU)."""
import numpy as np
import torch

from paper_2211_03516_gb300 import fins as F
from paper_2211_03516_gb300 import inputs as I


def test_fin_masks_cover_each_fin_once():
    w = I.fins_workload(3)
    f = I.make_target(w) > 0.5
    fins, gaps = F.fin_masks(w, 3)
    assert len(fins) == 3 and all(m.any() for m in fins)
    for m in fins:
        assert f[m].all()                       # a fin mask lies inside the part
    for g in gaps:
        assert g.any() and not f[g].any()       # a gap mask lies outside it
    assert not (fins[0] & fins[1]).any()


def test_fins_formed_counts():
    w = I.fins_workload(3)
    f = torch.from_numpy(I.make_target(w))
    fins, gaps = F.fin_masks(w, 3)
    idx = 512                                   # cure at half the maximum
    r = F.fins_formed(f.clone(), w, 3, idx)
    assert r["formed"] == 3 and all(p["fin_cured"] == 1.0 and p["gap_liquid"] == 1.0 for p in r["per_fin"])
    d = f.clone()
    d[torch.from_numpy(fins[1])] = 0.2          # fin 1 under-dosed
    d[torch.from_numpy(gaps[2])] = 0.9          # the gap above fin 2 over-dosed
    r = F.fins_formed(d, w, 3, idx)
    assert [p["formed"] for p in r["per_fin"]] == [True, False, False] and r["formed"] == 1
