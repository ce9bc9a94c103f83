"""iim_apply_noalloc: the operator without the problem's own ghost scratch.

Some callers cannot allocate device memory once their problems are set up: code that runs
under a fixed device-memory budget with nothing left to grow into, for instance.  For them
the library offers one entry point that writes its scratch (the ghost values) into a fixed
area compiled into the library instead of memory the problem allocated.  This file checks
it through the C ABI:

* against iim_apply, the regular entry point, on two calls in a row (the area keeps the
  previous call's contents, so the second call must not depend on them).  Both run the
  same kernels in the same order, so the results are compared bit for bit;
* against the oracle's operator, within the 1e-12 relative bound of the parity tests;
* a problem whose ghost values do not fit the area is refused with IIM_ERR_CAPACITY before
  anything is launched, and the output buffer is left as it was.

The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import workloads as W
from oracle.problem import OracleProblem
from tests.gpu_helpers import dev, gpu_problem, need_gpu, rel_err, set_gpu_data

pytestmark = pytest.mark.gpu

# the area's size in doubles (the limit stated in iim.h)
AREA_DOUBLES = 1 << 18


def _spec(case):
    if case == "interface":
        return W.star_interface_1024(128)
    return W.ProblemSpec(n=80, geometry=W.Geometry(W.ELLIPSE, (0.02, -0.03, 0.4, 0.3, 0.5), False),
                         bc=W.NEUMANN, order=6, box_bc=W.BOX_DIRICHLET, beta_plus=2.0,
                         solution=W.sin_cos_2d(2.0, 0.3, 1.5, 0.7))


@pytest.mark.parametrize("case", ["interface", "neumann"])
def test_noalloc_apply_matches_apply_on_two_calls(case):
    torch, iim = need_gpu()
    spec = _spec(case)
    P = gpu_problem(iim, spec)
    set_gpu_data(P, spec)
    rng = np.random.default_rng(21)
    for call, include_data in ((1, False), (2, True)):
        u = dev(rng.standard_normal(P.N))
        ref = P.apply(u, include_data=include_data).cpu().numpy()
        got = P.apply_noalloc(u, include_data=include_data).cpu().numpy()
        assert np.array_equal(got, ref), (call, rel_err(got, ref))


def test_noalloc_apply_matches_the_oracle():
    """The manufactured solution with the problem's data, as in the operator parity tests:
    L u + L_Gamma u_Gamma cancels down to the truncation error, so the difference is
    measured against the size of the terms summed (max |L u|)."""
    torch, iim = need_gpu()
    spec = _spec("interface")
    P = gpu_problem(iim, spec)
    set_gpu_data(P, spec)
    O = OracleProblem(spec)
    f, data = O.data()
    u = O.exact()
    ref = O.op.apply(u, data, include_data=True)
    scale = np.max(np.abs(O.op.apply(u)))
    for _ in range(2):
        got = P.apply_noalloc(dev(u), include_data=True).cpu().numpy()
        assert np.max(np.abs(got - ref)) < 1e-12 * scale


def test_noalloc_apply_refuses_a_problem_beyond_the_area():
    """A 256^3 sphere (4,5) has about 1.5e5 control points, so its ghost values (2 per
    control point) exceed the 2^18 doubles of the area."""
    torch, iim = need_gpu()
    spec = W.ProblemSpec(n=256, geometry=W.Geometry(W.SPHERE, (0.01, -0.02, 0.015, 0.7), True),
                         bc=W.DIRICHLET, order=4, solution=W.sin_sin_cos_3d((1.0, 2.0, 1.5), (0.1, 0.2, 0.3)))
    P = gpu_problem(iim, spec)
    nfit, _, _ = iim.fit_stats(P)
    assert nfit * 2 > AREA_DOUBLES
    u = dev(np.ones(P.N))
    w = dev(np.full(P.N, 7.0))
    with pytest.raises(iim.IIMError) as exc:
        P.apply_noalloc(u, out=w)
    assert exc.value.status == iim.IIM_ERR_CAPACITY
    torch.cuda.synchronize()
    assert bool(torch.all(w == 7.0))
    # the problem itself is unharmed: the regular entry point still works
    P.apply(u, out=w)
    assert bool(torch.isfinite(w).all())
