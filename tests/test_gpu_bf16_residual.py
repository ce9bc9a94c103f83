"""FP32 multigrid with the restricted residuals rounded to BF16 where they are stored.

The preconditioner changes (its coarse right-hand sides carry 8 significant
bits), the discrete system does not: the solve must reach the same unique
solution as the FP32 form (to the bound set by the tolerance), one V-cycle must
differ from the FP32 V-cycle by about BF16 rounding and no more, and the
iteration counts of both forms are reported for the 2D and 3D cases.
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import dev, gpu_problem, need_gpu, rel_err, set_gpu_data

pytestmark = pytest.mark.gpu

CASES = {
    "star_interface_6_256": lambda: W.star_interface_1024(256),
    "ellipsoid_neumann_4_64": lambda: W.ellipsoid_neumann_256(64),
}


@pytest.fixture(scope="module")
def env():
    return need_gpu()


@pytest.mark.parametrize("case", sorted(CASES))
def test_bf16_residual_form_reaches_the_same_solution(env, case, capsys):
    torch, iim = env
    spec = CASES[case]()
    out = {}
    for name, prec in (("fp32", iim.MG_FP32), ("bf16r", iim.MG_FP32_BF16R)):
        P = gpu_problem(iim, spec, tol=1e-12, mg_precision=prec)
        set_gpu_data(P, spec)
        x, info = P.solve()
        assert info.converged and info.relres <= 1e-12, (name, info.as_dict())
        v = np.random.default_rng(5).standard_normal(P.N)
        z = P.precondition(dev(v)).cpu().numpy()
        out[name] = (x.cpu().numpy(), info.iters, z)
        P.close()
    (x32, it32, z32), (x16, it16, z16) = out["fp32"], out["bf16r"]
    assert rel_err(x16, x32) < 1e-9
    dz = np.linalg.norm(z16 - z32) / np.linalg.norm(z32)
    assert 1e-6 < dz < 5e-2, dz
    with capsys.disabled():
        print(f"\n[{case}] FGMRES iterations to 1e-12: fp32 MG {it32}, bf16-residual MG {it16}; "
              f"one V-cycle differs by {dz:.2e}")
