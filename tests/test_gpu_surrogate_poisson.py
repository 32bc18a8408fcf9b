"""What the trained surrogate gains over the method without it, at the
Poisson solution error (the benchmark problem of Section 5 on the disk with
holes, u = sin(pi x) sin(pi y), one host sparse direct solve per weight set).

The interior Laplacian rows come from the surrogate (network -> projection
onto the monomial rows -> residual check rho <= tau -> FP32 + refinement
solve of the rejected stencils); the boundary d/dn rows from the FP32 +
refinement solve.  Measured trade-off, asserted here:
  * a strict check (tau = 1e-4) keeps the Poisson error within 1% of the
    FP64 weights' (what it accepts is as good as the solve) but accepts
    almost nothing, so it is no faster than the FP32 + refinement solve;
  * a loose check (tau = 1e-3) accepts most interior stencils and is faster
    than the FP32 + refinement solve on the same rows, at a Poisson error
    that is no longer equal to FP64's (the accepted weights carry the
    network's ~1% error).
So at equal Poisson error the surrogate gains nothing over the FP32 +
refinement solve with this network; its gain is speed at a larger error, and
only when the network is trained well enough to accept most stencils.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1912_13282_gb300 import _build
    _build.build()
    import paper_1912_13282_gb300 as P
    from paper_1912_13282_gb300 import surrogate as S
    ctx = P.Context(0)
    # the benchmark's network: 2^20 patch stencils, 120 epochs (a network
    # trained on 2^19 stencils for 80 epochs accepted fewer stencils and was
    # no faster than the solve even at tau = 1e-3)
    data = S.make_dataset(ctx, 1 << 20, seed=1)
    net = P.MLP(ctx, 50, 25, seed=0)
    S.train(net, data["x"], data["t"], epochs=120, batch=4096, lr=3e-3, lr_final=1e-4)
    del data
    yield P, ctx, net
    net.close()
    ctx.close()


def test_surrogate_tradeoff_at_poisson_error(setup):
    import bench
    P, ctx, net = setup
    res = bench.surrogate_poisson(P, ctx, net, (1e-3, 1e-4), n_target=100_000, reps=5)
    f = res["forms"]
    e64 = f["fp64"]["poisson_max_error"]
    assert 1e-8 < e64 < 1e-5, e64                      # the discretisation error of this node set
    assert f["fp32_ir"]["equal_within_1pct"], f["fp32_ir"]
    strict, loose = f["surrogate_tau_0.0001"], f["surrogate_tau_0.001"]
    # strict check: equal Poisson error, nearly everything solved
    assert strict["equal_within_1pct"], strict
    assert strict["accept_fraction"] < 0.2, strict
    # loose check: most stencils accepted and faster than the solve
    assert loose["accept_fraction"] > 0.4, loose
    assert loose["interior_weights_ms"] < f["fp32_ir"]["interior_weights_ms"], (loose, f["fp32_ir"])
    assert np.isfinite(loose["poisson_max_error"]) and loose["poisson_max_error"] < 10 * e64, loose
