"""The oracle's pins must catch plausible mistakes. Each case plants one
mistake in a copy of oracle/nb_oracle.c (on the CPU), compiles it, and runs
the CPU pin tests against that copy: at least one pin must fail. The
replacement must match the source exactly once, so a case fails loudly if
the source changes under it."""
import inspect
import os

import pytest

import oracle
import test_oracle_dynamics as dyn
import test_oracle_force as frc

SRC = os.path.join(os.path.dirname(oracle.__file__), "nb_oracle.c")

MUTATIONS = {
    "self_term_included": ("        if (j == i) continue;\n", "\n"),
    "exponent_s_minus_1": ("inv_s32 = inv_sqrt_s * inv_sqrt_s * inv_sqrt_s;",
                           "inv_s32 = inv_sqrt_s * inv_sqrt_s;"),
    "difference_sign": ("const double dx = xi - x[3 * j + 0];",
                        "const double dx = x[3 * j + 0] - xi;"),
    "target_mass": ("ax += m[j] * dx * inv_s32;", "ax += m[i] * dx * inv_s32;"),
    "eps_not_squared": ("double eps,\n               double *a, double *p, double *amag)\n{\n"
                        "    const double eps2 = eps * eps;",
                        "double eps,\n               double *a, double *p, double *amag)\n{\n"
                        "    const double eps2 = eps;"),
    "transposed_component": ("const double dy = yi - x[3 * j + 1];",
                             "const double dy = yi - x[3 * j + 2];"),
    "potential_power": ("pp += m[j] * inv_sqrt_s;", "pp += m[j] * inv_sqrt_s * inv_sqrt_s;"),
    "vjp_missing_partner_half": ("gx0 -= m[k] *", "gx0 -= 0.0 * m[k] *"),
    "vjp_mass_gradient_sign": ("gmm += -rgl * sm32 + gp[l] * sm12;",
                               "gmm += rgl * sm32 + gp[l] * sm12;"),
    "vjp_factor_three": ("gx1 += m[l] * (sm32 * ga[3 * k + 1] - 3.0 * sm52",
                         "gx1 += m[l] * (sm32 * ga[3 * k + 1] - 2.0 * sm52"),
    "leapfrog_repulsive_kick": ("const double g0 = -a[k];", "const double g0 = a[k];"),
    "leapfrog_full_kick": ("v[k] = v0 + 0.5 * g0 * dt;", "v[k] = v0 + g0 * dt;"),
    "leapfrog_drift_without_half": ("x[k] = x[k] + v0 * dt + 0.5 * g0 * dt * dt;",
                                    "x[k] = x[k] + v0 * dt + g0 * dt * dt;"),
    "energy_double_counted_pairs": ("pot += -0.5 * m[i] * p[i];", "pot += -m[i] * p[i];"),
}


def _pins():
    """Every CPU pin test of the oracle, as (name, callable taking the oracle)."""
    out = []
    for mod in (frc, dyn):
        for name, fn in inspect.getmembers(mod, inspect.isfunction):
            if not name.startswith("test_"):
                continue
            params = list(inspect.signature(fn).parameters)
            marks = getattr(fn, "pytestmark", [])
            cases = [m.args for m in marks if m.name == "parametrize"]
            if params == ["oracle_mod"]:
                out.append((name, lambda o, fn=fn: fn(o)))
            elif params == ["oracle_mod", "case", "vals"] and cases:
                for case, vals in cases[0][1]:
                    out.append((f"{name}[{case}]", lambda o, fn=fn, c=case, v=vals: fn(o, c, v)))
    return out


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    pytest.importorskip("mpmath")
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation {name} does not match the oracle source exactly once"
    mutated = tmp_path / "nb_oracle_mutated.c"
    mutated.write_text(src.replace(old, new))
    lib = oracle.build(force=True, src=str(mutated), out=str(tmp_path / "libmut.so"))
    mut = oracle.Oracle(lib)
    failed = []
    for pin, run in _pins():
        try:
            run(mut)
        except (AssertionError, FloatingPointError, ZeroDivisionError):
            failed.append(pin)
    assert failed, f"no pin caught the planted mistake {name}"


# Planted mistakes in the reverse-mode trajectory gradient (Python, oracle.Oracle.
# leapfrog_grad): each must make its central-difference pin fail.
PY_MUTATIONS = {
    "grad_back_kick_sign": ("ab_next = ab - 0.5 * dt * vb", "ab_next = ab + 0.5 * dt * vb"),
    "grad_drift_dt2_term": ("ab = -0.5 * dt * vb - 0.5 * dt * dt * xb", "ab = -0.5 * dt * vb"),
    "grad_drift_half_dt": ("vb = vb + dt * xb", "vb = vb + 0.5 * dt * xb"),
    "grad_force_at_step_start": ("self.force_vjp(xs[s + 1], m, eps, ab_next, zero_p)",
                                 "self.force_vjp(xs[s], m, eps, ab_next, zero_p)"),
    "grad_mass_term_dropped": ("mb = mb + gm\n", "mb = mb\n"),
    "grad_first_force_dropped": ("return xb + gx, vb, mb + gm", "return xb, vb, mb"),
}


def _mutated_grad_oracle(old, new):
    import textwrap
    import types
    src = textwrap.dedent(inspect.getsource(oracle.Oracle.leapfrog_grad))
    if old:
        assert src.count(old) == 1, f"mutation does not match leapfrog_grad exactly once: {old!r}"
        src = src.replace(old, new)
    ns = dict(vars(oracle))
    exec(compile(src, "<mutated leapfrog_grad>", "exec"), ns)
    inst = oracle.Oracle()
    inst.leapfrog_grad = types.MethodType(ns["leapfrog_grad"], inst)
    return inst


@pytest.mark.parametrize("name", sorted(PY_MUTATIONS))
def test_planted_gradient_mistake_is_caught(name):
    mut = _mutated_grad_oracle(*PY_MUTATIONS[name])
    with pytest.raises(AssertionError):
        dyn.test_leapfrog_grad_matches_central_differences(mut)


def test_unmutated_gradient_copy_passes():
    # The harness itself: the method re-executed unchanged passes its pin.
    dyn.test_leapfrog_grad_matches_central_differences(_mutated_grad_oracle("", ""))


def test_unmutated_copy_passes_every_pin(tmp_path):
    # The harness itself: an unchanged copy built the same way passes.
    lib = oracle.build(force=True, src=SRC, out=str(tmp_path / "libcopy.so"))
    copy = oracle.Oracle(lib)
    for pin, run in _pins():
        run(copy)
