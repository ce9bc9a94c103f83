"""iim_apply_noalloc: the operator without the problem's own ghost scratch.

For callers that cannot allocate device memory once their problems are set up
(a fixed memory budget, or work recorded while a stream is captured), the
library offers one entry point that writes its scratch into a fixed area
compiled into the library instead.  This checks it through the C ABI against
iim_apply, the regular entry point, on two calls in a row (the area keeps the
previous call's contents, so the second call must not depend on them).
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import dev, gpu_problem, need_gpu, rel_err, set_gpu_data

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["interface", "neumann"])
def test_noalloc_apply_matches_apply_on_two_calls(case):
    torch, iim = need_gpu()
    if case == "interface":
        spec = W.star_interface_1024(128)
    else:
        spec = W.ProblemSpec(n=80, geometry=W.Geometry(W.ELLIPSE, (0.02, -0.03, 0.4, 0.3, 0.5), False),
                             bc=W.NEUMANN, order=6, box_bc=W.BOX_DIRICHLET, beta_plus=2.0,
                             solution=W.sin_cos_2d(2.0, 0.3, 1.5, 0.7))
    P = gpu_problem(iim, spec)
    set_gpu_data(P, spec)
    rng = np.random.default_rng(21)
    for call, include_data in ((1, False), (2, True)):
        u = dev(rng.standard_normal(P.N))
        ref = P.apply(u, include_data=include_data).cpu().numpy()
        got = P.apply_noalloc(u, include_data=include_data).cpu().numpy()
        assert rel_err(got, ref) < 1e-12, (call, rel_err(got, ref))
