"""What the FP32 rounding of the device's parameters does to an inlet-driven
artery run, in the FP64 oracle: the odd TRT rate rounded to FP32 and the
inlet velocities perturbed by 1e-7 relative (more than the FP32 rounding of
the inlet map constants) each move the velocity field by far less than the
~1e-5 that separates the FP32 device run of the full tree from the FP64
oracle.  So that gap is the FP32 arithmetic acting through the pressurising
transient, not a mismatch of parameters, and the artery's parity bound is
set by it rather than by the inputs."""
import numpy as np

import geometry as G
import oracle as O


class _RoundedOdd(O.Problem):
    """The oracle's problem with the odd TRT rate replaced by a given value."""
    om_override = None

    @property
    def omega_minus(self):
        return self.om_override if self.om_override is not None else super().omega_minus


def _run(g, steps, om=None, inlet_scale=1.0):
    gi = G.Geometry(g.flags, g.periodic, g.inlet_u * inlet_scale, g.rho_out, g.meta)
    p = _RoundedOdd.from_geometry(gi, q=19, op=O.TRT, omega_plus=1.25, magic=3 / 16, force=(0.0, 0.0, 0.0))
    p.om_override = om
    L = O.pull_list(p)
    return O.sparse_macroscopic(p, L, O.sparse_run(p, L, O.sparse_rest(p, L), steps))


def test_parameter_rounding_moves_an_artery_run_far_less_than_fp32_arithmetic():
    g = G.artery_tree(256, 128, 128, r0=6.0, r_leaf=2.0)
    steps = 400
    rho0, u0 = _run(g, steps)
    assert rho0.max() > 1.001                                  # the inlet pressurises the tree
    om = O.trt_omega_minus(1.25, 3 / 16)
    om32 = float(np.float32(om))
    assert om32 != om
    _, u1 = _run(g, steps, om=om32)
    _, u2 = _run(g, steps, inlet_scale=1 + 1e-7)
    n = np.linalg.norm(u0)
    # measured here 2.5e-10 and 9.8e-8 (29 767 cells, 400 steps); on the tree
    # at 512 x 256 x 256 after 2000 steps 1.3e-10 and 9.8e-8, while the FP32
    # device run of the full tree differs from the oracle by 1.2e-5
    assert np.linalg.norm(u1 - u0) / n < 1e-8
    assert np.linalg.norm(u2 - u0) / n < 5e-7
