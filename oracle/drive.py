"""Driven optimisation of the penalty coefficient, written plainly.  Test
infrastructure only.

Methods, "Numerical Convergence": the link constraint L = 2 is imposed by
the penalty nu sum (1 - delta_{2,L}) of Eq. (16).  A large nu from the first
sweep can trap the variational search, so nu is driven in three stages:
  (i)   from a small value and a random state, nu grows linearly from sweep
        to sweep until the energy starts to go up;
  (ii)  then nu grows quadratically, so that in the sweeps right after the
        switch the increments are smaller than in the linear stage;
  (iii) once nu reaches the wanted maximum it stays there, and sweeps run
        until the energy has converged.
Methods, "Tensor Networks": the precision of the local eigensolver is
raised from sweep to sweep.  delta_L = sum over links |<L - 2>| (the
definition after Eq. (16)) is recorded after every sweep.

Readings of what the paper leaves open (none of these numbers is given):
  - "rise": the energy <H + H_pen> after a sweep of the linear stage
    exceeds the one after the sweep before it by more than rise_rel times
    the latter's magnitude (so that rounding does not count as a rise); the
    sweep that shows it is the last linear one and its nu is the start of
    the quadratic stage;
  - quadratic stage: the k-th sweep after the switch has
    nu = nu_switch + quad_coef * nu_step * k**2 (quad_coef < 1 gives first
    increments below nu_step);
  - a stage whose next nu would reach nu_max stops there, and every later
    sweep uses nu_max;
  - converged: at least min_final_sweeps sweeps at nu_max, and the last two
    energies differ by at most conv_rel |E|;
  - tolerance of sweep s: max(tol_final, tol_start * tol_factor**s).
"""


class Schedule:
    """Penalty and tolerance of each sweep from the energies seen so far."""

    def __init__(self, nu_start, nu_step, quad_coef, nu_max, tol_start, tol_factor, tol_final, conv_rel,
                 rise_rel, min_final_sweeps):
        self.nu_step = nu_step
        self.quad_coef = quad_coef
        self.nu_max = nu_max
        self.tol_start = tol_start
        self.tol_factor = tol_factor
        self.tol_final = tol_final
        self.conv_rel = conv_rel
        self.rise_rel = rise_rel
        self.min_final = min_final_sweeps
        self.history = []            # (nu, stage, energy) of the sweeps run
        self.nu_switch = None
        self.k_since_switch = 0
        self.next_nu = min(nu_start, nu_max)
        self.next_stage = "constant" if nu_start >= nu_max else "linear"
        self.converged = False

    def tol(self):
        s = len(self.history)
        return max(self.tol_final, self.tol_start * self.tol_factor ** s)

    def record(self, energy):
        """The sweep with (next_nu, next_stage) ended at `energy`."""
        nu, stage = self.next_nu, self.next_stage
        prev = self.history[-1][2] if self.history else None
        self.history.append((nu, stage, energy))
        if stage == "constant":
            at_max = sum(1 for h in self.history if h[1] == "constant")
            if at_max >= self.min_final and abs(energy - prev) <= self.conv_rel * abs(energy):
                self.converged = True
            return
        if stage == "linear":
            if prev is not None and energy - prev > self.rise_rel * abs(prev):
                self.nu_switch = nu
                self.k_since_switch = 1
                want, new_stage = nu + self.quad_coef * self.nu_step * 1 ** 2, "quadratic"
            else:
                want, new_stage = nu + self.nu_step, "linear"
        else:
            self.k_since_switch += 1
            k = self.k_since_switch
            want, new_stage = self.nu_switch + self.quad_coef * self.nu_step * k ** 2, "quadratic"
        if want >= self.nu_max:
            want, new_stage = self.nu_max, "constant"
        self.next_nu, self.next_stage = want, new_stage


STAGE_CODE = {"linear": 0, "quadratic": 1, "constant": 2}


def run(state, nu_start, nu_step, quad_coef, nu_max, tol_start, tol_factor, tol_final, conv_rel, rise_rel,
        min_final_sweeps, max_sweeps):
    """Driven sweeps of an oracle TTN: before each sweep the penalty is set
    to the schedule's nu (when it changed), one sweep at the schedule's
    tolerance, then the energies at the root and delta_L.  Returns
    (records, converged)."""
    sch = Schedule(nu_start, nu_step, quad_coef, nu_max, tol_start, tol_factor, tol_final, conv_rel, rise_rel,
                   min_final_sweeps)
    records = []
    while not sch.converged and len(records) < max_sweeps:
        nu, stage, tol = sch.next_nu, sch.next_stage, sch.tol()
        if state.p.nu != nu:
            state.set_couplings(nu=nu)
        state.sweep(tol)
        state.move_to(len(state.nodes) - 1)
        e = state.energy_at_center()
        obs = state.observables()
        e_pen = _penalty_energy(state)
        records.append({"sweep": len(records), "stage": STAGE_CODE[stage], "nu": nu, "tol": tol, "energy": e,
                        "energy_without_penalty": e - e_pen, "delta_L": obs["delta_L"]})
        sch.record(e)
    return records, sch.converged


def _penalty_energy(state):
    """<H_pen> of the state: the expectation of the penalty terms alone."""
    from . import model as _model
    from . import ttn as _ttn
    return _ttn.expectation(state, _model.class_only(state.p, "nu"))
