"""FE² on the GPU: a two-element strip with one RVE per Gauss point (FP64
tangents); the macroscale Newton converges and the stress grows with load."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe2mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2306_09427_gb300 import fe2
    return fe2


def test_strip_newton_converges(fe2mod):
    import paper_2306_09427_gb300 as rve
    box = fe2mod.HexBox(1, 1, 2, 1.0, 1.0, 2.0)
    mat = fe2mod.RveMaterial(box.ne * 8, rve_side=5, p=0.7, precision=rve.RVE_PREC_BATCHED_F64, tol=1e-10)
    fe = fe2mod.FE2(box, mat)
    hist = fe.run(strain=0.02, steps=2, newton_tol=1e-7, max_newton=10, log=lambda *a: None)
    for h in hist:
        assert h["newton"][-1] <= 1e-7, h["newton"]
    assert 0 < hist[0]["reaction_z"] < hist[1]["reaction_z"]
    assert hist[1]["sigma_zz_mean"] > hist[0]["sigma_zz_mean"] > 0
    # the top moved by the prescribed stretch (the lateral faces are free)
    top = np.isclose(box.X[:, 2], 2.0)
    assert np.allclose(fe.u[top, 2], 0.04)
    mat.batch.close()


def test_strip_mixed_rves_match_fp64_rves(fe2mod):
    """The FE² answer with mixed-precision RVEs (their tangents are FP32
    stresses differenced over 2h = 2e-4, a few percent off) against the same
    strip with FP64 RVEs: the tangent only steers the macroscale Newton, so
    the converged reactions and stresses agree to the RVE stress accuracy."""
    import paper_2306_09427_gb300 as rve
    out = {}
    for name, prec, tol in (("mixed", rve.RVE_PREC_MIXED, 1e-7), ("fp64", rve.RVE_PREC_BATCHED_F64, 1e-10)):
        box = fe2mod.HexBox(1, 1, 2, 1.0, 1.0, 2.0)
        mat = fe2mod.RveMaterial(box.ne * 8, rve_side=5, p=0.7, precision=prec, tol=tol)
        fe = fe2mod.FE2(box, mat)
        out[name] = fe.run(strain=0.02, steps=2, newton_tol=1e-7, max_newton=20, log=lambda *a: None)
        mat.batch.close()
    for hm, hd in zip(out["mixed"], out["fp64"]):
        assert hm["newton"][-1] <= 1e-7 and hd["newton"][-1] <= 1e-7
        for key in ("reaction_z", "sigma_zz_mean"):
            d = abs(hm[key] - hd[key]) / abs(hd[key])
            print(f"step: {key} mixed {hm[key]:.10e} fp64 {hd[key]:.10e} rel {d:.2e}; Newton iterations "
                  f"{len(hm['newton'])} (mixed) / {len(hd['newton'])} (fp64)")
            assert d <= 1e-4, (key, d)
