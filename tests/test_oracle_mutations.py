"""Plant plausible mistakes in a copy of the oracle (CPU only) and check that
the pins of test_oracle_pins catch every one of them: a dropped term, a wrong
sign, a wrong index, a transposed operand, a misplaced tap, a swapped weight
or a dropped square in the loss."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import test_oracle_pins as pins
from gridcases import random_grid, three_bus_plus

MUTATIONS = {
    # Alg. 1's printed sign instead of Eq. (3)
    "alg1_sign": ("dth += I * V[i] * conj(Ib[i]);", "dth -= I * V[i] * conj(Ib[i]);"),
    # dropped diagonal term of Eq. (4)
    "drop_diag_dv": ("dv += conj(Ib[i]) * U[i];", "dv += 0.0 * conj(Ib[i]) * U[i];"),
    # transposed operand: V_i instead of V_j inside the conjugate
    "transpose_dth": ("cplx dth = -I * V[i] * conj(Y * V[j]);", "cplx dth = -I * V[i] * conj(Y * V[i]);"),
    # phase-shift sign of the h-k coupling stamp
    "shift_sign": ("cplx yhk = -ys * eph / m;", "cplx yhk = -ys * conj(eph) / m;"),
    # tap applied once instead of squared on the primary self-admittance
    "tap_power": ("cplx yhh = (ys + ysh) / (m * m);", "cplx yhh = (ys + ysh) / m;"),
    # wrong magnitude index in a partial of the element-wise method
    "ew_index": ("p[3] = Xh / vk;", "p[3] = Xh / vh;"),
    # wrong angle sign in the k-terminal flow
    "ew_angle": ("cplx Xk = -vh * vk * conj(yhk) / m * cexp(-I * (d - shift[l]));",
                 "cplx Xk = -vh * vk * conj(yhk) / m * cexp(-I * (d + shift[l]));"),
    # bus shunt dropped from the element-wise reduction
    "ew_shunt": ("cplx S = vm[i] * vm[i] * conj(ysh);", "cplx S = 0.0 * conj(ysh);"),
    # residual weight mix-up in the adjoint
    "adj_weight": ("double rQ = 2.0 * wQ[i] * (Q[i] - Qs[i]);", "double rQ = 2.0 * wP[i] * (Q[i] - Qs[i]);"),
    # transposed Jacobian in J^T r
    "adj_transpose": ("gva[j] += J[p] * rP + J[2 * nnz + p] * rQ;", "gva[i] += J[p] * rP + J[2 * nnz + p] * rQ;"),
    # P and Q weights swapped in the loss
    "loss_weight_swap": ("double dp = P[i] - Ps[i], dq = Q[i] - Qs[i];\n        L += wP[i] * dp * dp + wQ[i] * dq * dq;",
                         "double dp = P[i] - Ps[i], dq = Q[i] - Qs[i];\n        L += wQ[i] * dp * dp + wP[i] * dq * dq;"),
    # a dropped square in the loss
    "loss_square": ("double dp = P[i] - Ps[i], dq = Q[i] - Qs[i];\n        L += wP[i] * dp * dp + wQ[i] * dq * dq;",
                    "double dp = P[i] - Ps[i], dq = Q[i] - Qs[i];\n        L += wP[i] * dp + wQ[i] * dq * dq;"),
}


def _all_pins():
    errs = {
        "two_bus": pins.pin_two_bus(),
        "circuit_3bus": pins.pin_circuit_law(three_bus_plus()),
        "circuit_shift": pins.pin_circuit_law(random_grid(120, 170, 11, shift_max=0.3)),
        "cstep": pins.pin_jacobian_cstep(random_grid(120, 170, 31, shift_max=0.3)),
        "invariants": pins.pin_invariants(three_bus_plus()),
        "ew_eq_ybus": pins.pin_elementwise_equals_ybus(random_grid(120, 170, 51, shift_max=0.3)),
        "ew_eq_ybus_3": pins.pin_elementwise_equals_ybus(three_bus_plus()),
        "branch_loss": pins.pin_branch_loss(),
        "adjoint": pins.pin_adjoint(60, 80, 7),
        "loss_closed": pins.pin_loss_closed_form(),
        "loss_fd": pins.pin_loss_central_difference(60, 80, 7),
    }
    return errs


LIMITS = {"two_bus": 1e-14, "branch_loss": 1e-12, "adjoint": 1e-8, "loss_closed": 1e-14, "loss_fd": 1e-6}


def test_unmutated_oracle_passes_all_pins():
    errs = _all_pins()
    bad = {k: v for k, v in errs.items() if not v < LIMITS.get(k, 1e-13)}
    assert not bad, bad


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, tmp_path):
    src = open(oracle.SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, "mutation anchor not found exactly once: %s" % old
    path = tmp_path / "oracle_mut.c"
    path.write_text(src.replace(old, new))
    lib_path = str(tmp_path / "liboracle_mut.so")
    cc = shutil.which("gcc") or "cc"
    subprocess.check_call([cc, "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-o", lib_path,
                           str(path), "-lm"])
    saved = oracle._lib
    try:
        oracle._lib = oracle.bind(lib_path)
        errs = _all_pins()
    finally:
        oracle._lib = saved
    caught = {k: v for k, v in errs.items() if not (v < LIMITS.get(k, 1e-13)) or not np.isfinite(v)}
    assert caught, "mutation %s survived every pin: %s" % (name, errs)
