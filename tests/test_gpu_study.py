"""The study drivers (paper_1612_08792_gb300.study) run end to end on small cases."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def study():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1612_08792_gb300 import study
    torch.cuda.set_device(0)
    return study


def test_sweep_rows(study):
    rows = study.sweep("eps_c", values=(2, 8), spacings=(15, 30), n_images=3, iters=3, batch=2)
    assert [(r["spacing"], r["eps_c"]) for r in rows] == [(15, 2.0), (15, 8.0), (30, 2.0), (30, 8.0)]
    for r in rows:
        assert 0.0 <= r["ue"] <= 1.0 and 0.5 <= r["asa"] <= 1.0 and 0.0 <= r["br"] <= 1.0
        assert r["images"] == 3 and r["loglik_per_pixel"] < 0
    # a higher colour floor bounds the colour densities from above: lower likelihood
    assert rows[1]["loglik_per_pixel"] < rows[0]["loglik_per_pixel"]
    rows = study.sweep("lambda_c", values=(4,), spacings=(20,), n_images=2, iters=2)
    assert rows[0]["lambda_c"] == 4.0 and rows[0]["K"] == (481 // 20) * (321 // 20)


def test_colour_models_summary(study):
    res = study.colour_models(n_images=4, iters=3, reps=1)
    assert set(res["models"]) == {"full", "split", "gray"}
    m = res["models"]
    for r in m.values():
        assert r["mpix_per_s"] > 0 and 0.5 <= r["asa"] <= 1.0
    # the split family is a subset of the full one: it fits no better
    assert m["split"]["loglik_per_pixel"] < m["full"]["loglik_per_pixel"]
