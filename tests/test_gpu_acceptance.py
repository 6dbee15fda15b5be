"""Acceptance on the 3D deformed cube (p = 3, manufactured load, tol 1e-8),
at n = 48 and n = 64: the GPU solutions against the FP64 oracle's own solve
of the same problem (its own A and b, assembled on the host). The full
n = 128 workload (2,097,152 dofs) is checked the same way by the benchmark's
oracle leg (its vs_oracle entry), whose host assembly takes minutes.

Readings of the targets (O17): the all-FP64 path runs the oracle's
algorithm, so at the same tolerance it stops at the same iteration and its
iterate matches the oracle's to 1e-10 (entry-wise and in the 2-norm); the
mixed-precision FD (TF32 tensor cores) converges to the same discrete
solution, so its 1e-8 solution matches the oracle's 1e-13 one to 1e-7, with
at most two more iterations than the FP64 preconditioner.
"""
import numpy as np
import pytest

import synth
from gpu_util import need_gpu, rel, maxrel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [48, 64])
def test_solution_matches_oracle(n):
    torch = need_gpu()
    import bench
    from paper_1602_01636_gb300 import igafd
    o = bench.OracleRun(n, 3)
    res8, _, _ = o.solve(1e-8)
    res13, _, _ = o.solve(1e-13, x0=res8.x, max_iter=3 * res8.iters + 20)
    assert res8.converged and res13.true_relres <= 1e-11
    patch = igafd.Patch.from_problem(synth.deformed_cube(n, 3, seed=0))
    b = patch.load_rhs_sine()
    assert maxrel(b.cpu().numpy(), o.b) <= 1e-13
    x64, i64 = patch.pcg(b, tol=1e-8, dtype="fp64")
    xtf, itf = patch.pcg(b, tol=1e-8, dtype="tf32")
    patch.close()
    x64, xtf = x64.cpu().numpy(), xtf.cpu().numpy()
    e64, e64_l2 = maxrel(x64, res8.x), rel(x64, res8.x)
    etf, etf_l2 = maxrel(xtf, res13.x), rel(xtf, res13.x)
    print(f"n={n}: oracle {res8.iters} it (+{res13.iters} to 1e-13); GPU FP64 {i64.iterations} it, "
          f"vs oracle {e64:.2e} (2-norm {e64_l2:.2e}); TF32 {itf.iterations} it, vs converged "
          f"{etf:.2e} (2-norm {etf_l2:.2e}); FP64 vs converged {maxrel(x64, res13.x):.2e}")
    assert i64.status == 0 and itf.status == 0
    assert i64.iterations == res8.iters
    assert e64 <= 1e-10 and e64_l2 <= 1e-10
    assert etf <= 1e-7 and etf_l2 <= 1e-7
    assert itf.iterations <= i64.iterations + 2
