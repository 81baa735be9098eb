"""The optimisation loop of Sec. "Parallel optimization procedure" on a small cantilever:
material decreases, compliance rises, the supports and loads stay, every BVP converges to
the FP64 residual, and the design stays connected to the supports."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def K():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_04082_gb300 as K
    return K


def test_cantilever_iterations(K):
    from paper_1612_04082_gb300 import driver as D
    prob = D.cantilever(6)  # 12 x 6 x 6 voxels, 1/6 cells
    mask, hist = D.optimize(prob, C=0.02, iters=4)
    assert len(hist) >= 3
    alphas = [h.stats["alpha"] for h in hist]
    psis = [h.stats["psi"] for h in hist]
    assert all(a > b for a, b in zip(alphas, alphas[1:]))
    assert all(b > a for a, b in zip(psis, psis[1:]))  # less material, more compliant
    assert psis[0] > 0
    for h in hist:
        assert h.stats["converged"] and h.stats["relres"] <= 1e-6
        assert h.features.shape == (h.stats["nt"], 11) and h.unknowns.shape == (h.stats["nt"], 3)
    frozen = prob.frozen()
    assert (mask[frozen > 0] == 1).all()
    # connected to the supports: cleaning removes nothing more
    m2 = mask.copy()
    assert K.voxel_clean(m2, prob.support) == 0
    # carried-over unknowns: faces that survive keep their previous values in the features
    f1 = hist[1].features
    assert np.abs(f1[:, 7:10]).sum() > 0


def test_previous_iterate_start_cuts_iterations(K):
    """Starting the next BVP from the previous iterate (carried over by face identity) needs
    fewer inner GMRES iterations than starting from zero."""
    from paper_1612_04082_gb300 import driver as D
    prob = D.cantilever(6)
    _, cold = D.optimize(prob, C=0.02, iters=3)
    _, warm = D.optimize(prob, C=0.02, iters=3, warm_start=lambda f: f[:, 7:10])
    assert sum(h.stats["iters"] for h in warm[1:]) < sum(h.stats["iters"] for h in cold[1:])


def test_learned_warm_start_beats_zero_start(K):
    """The network trained on the earlier iterations gives initial guesses from which the
    later BVPs need fewer inner GMRES iterations than from zero (same designs, same
    tolerance: the FP64 residual of 1e-6)."""
    from paper_1612_04082_gb300 import driver as D
    prob = D.cantilever(6)
    _, cold = D.optimize(prob, C=0.02, iters=4)
    ws = D.LearnedWarmStart()
    _, warm = D.optimize(prob, C=0.02, iters=4, warm_start=ws)
    assert [h.stats["nt"] for h in warm] == [h.stats["nt"] for h in cold]
    assert all(h.stats["converged"] for h in warm)
    later_cold = sum(h.stats["iters"] for h in cold[2:])
    later_warm = sum(h.stats["iters"] for h in warm[2:])
    assert later_warm < later_cold
    ws.net.close()


def test_adaptive_td_sampling_gives_the_same_designs(K):
    """Two-scale D^T sampling (Sec. "Discussion and future work") against D^T at every
    material voxel: the same voxels removed at every iteration, so the same designs, with fewer
    D^T evaluations."""
    from paper_1612_04082_gb300 import driver as D
    prob = D.cantilever(6)
    m_full, full = D.optimize(prob, C=0.02, iters=4)
    m_ad, ad = D.optimize(prob, C=0.02, iters=4, td_sampling="adaptive")
    assert np.array_equal(m_full, m_ad)
    assert [h.stats["nt"] for h in full] == [h.stats["nt"] for h in ad]
    assert sum(h.stats["td_points"] for h in ad) < sum(h.stats["td_points"] for h in full)


def test_learned_start_against_previous_iterate_start(K):
    """The learned warm start against the previous-iterate start it builds on (the fair
    baseline, not a zero start); the measured counts are printed.  The network's direction is
    kept when it lowers the FMM residual of the new problem by 10%, which does not bound the
    GMRES iterations that follow: measured at this size, the later solves took 524 inner
    iterations against 451 (one solve 342 against 279).  The bound below catches a broken
    network (whose starts would cost far more) without asserting a gain the method does not
    have; whether it gains is a measurement, not a claim."""
    from paper_1612_04082_gb300 import driver as D
    prob = D.cantilever(6)
    _, prev = D.optimize(prob, C=0.02, iters=5, warm_start=lambda f: f[:, 7:10])
    ws = D.LearnedWarmStart()
    _, learned = D.optimize(prob, C=0.02, iters=5, warm_start=ws)
    assert [h.stats["nt"] for h in learned] == [h.stats["nt"] for h in prev]
    it_prev = [h.stats["iters"] for h in prev]
    it_learned = [h.stats["iters"] for h in learned]
    print("inner iterations, previous-iterate start:", it_prev, "learned start:", it_learned)
    assert sum(it_learned[2:]) <= 1.3 * sum(it_prev[2:])
    ws.net.close()
