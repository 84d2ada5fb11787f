"""Why an inlet-driven artery run in FP32 departs from the FP64 oracle by
~1e-5 after 2000 steps.  (1) Parameters: in the oracle, the odd TRT rate
rounded to FP32 and the inlet velocities perturbed by 1e-7 relative (more
than the FP32 rounding of the inlet map constants) each move the velocity
field by far less.  (2) Arithmetic: the same stepper over shifted
populations in float32 (tests/shifted_emulation.py; in float64 it is the
oracle to 1e-11) drifts from FP64 by more than 1e-5, growing with the step
count.  So the gap belongs to FP32 storage and arithmetic acting through the
pressurising transient, not to a mismatch of parameters."""
import numpy as np

import geometry as G
import oracle as O
import shifted_emulation as E


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


def _small_tree():
    g = G.artery_tree(256, 128, 128, r0=6.0, r_leaf=2.0)
    p = O.Problem.from_geometry(g, q=19, op=O.TRT, omega_plus=1.25, magic=3 / 16, force=(0.0, 0.0, 0.0))
    return p, O.pull_list(p)


def test_shifted_emulation_in_float64_is_the_oracle():
    p, L = _small_tree()
    rho_o, u_o = O.sparse_macroscopic(p, L, O.sparse_run(p, L, O.sparse_rest(p, L), 60))
    rho, u = E.run(p, L, 60, np.float64)
    assert np.linalg.norm(u - u_o) / np.linalg.norm(u_o) < 1e-11
    assert np.max(np.abs(rho - rho_o)) < 1e-12


def test_float32_shifted_populations_alone_drift_past_1e_5():
    # measured 6.2e-6 after 1000 steps and 1.35e-5 after 2000 (the FP32
    # device run of the same tree: 6.4e-6 and 1.24e-5)
    p, L = _small_tree()
    f = O.sparse_rest(p, L)
    errs = []
    emulated = E.run(p, L, (1000, 2000), np.float32)
    for (_, u), f_steps in zip(emulated, (1000, 1000)):
        f = O.sparse_run(p, L, f, f_steps)
        _, u_o = O.sparse_macroscopic(p, L, f)
        errs.append(np.linalg.norm(u - u_o) / np.linalg.norm(u_o))
    assert errs[1] > 1e-5
    assert 1.5 < errs[1] / errs[0] < 2.5                    # growing about linearly with the steps
