"""The oracle's stencils against the weights the paper prints (Sect. 2.3,
Eqs. 6-8; tests/golden/stencil_weights.txt).

Each weight is read back from the oracle by applying it to a unit impulse,
once through the point stencils (7 samples, a 7 x 7 patch) and once through
the periodic grid operators on every axis and axis pair, where the position
of each response also pins the index direction (a sign or a transposed
operand shows up as a weight in the wrong place).  The spacings are unequal
and not 1, so that the powers of the spacing in the prefactors are pinned
too."""
import os

import numpy as np
import pytest

from oracle import fd

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "stencil_weights.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].split()
        if line:
            out[line[0]] = (float(line[1]), [float(v) for v in line[2:]])
    return out


G = _golden()
TOL = 1e-10


def test_golden_file_is_complete():
    assert len(G["d1"][1]) == 7 and len(G["d2"][1]) == 7 and len(G["dmix"][1]) == 3


H = 0.37  # a spacing that is not 1, so that a missing power of it shows


@pytest.mark.parametrize("name, op", [("d1", fd.d1_point), ("d2", fd.d2_point)])
def test_point_stencil_weights(name, op):
    den, w = G[name]
    p = 1 if name == "d1" else 2
    for k in range(-3, 4):
        e = np.zeros(7)
        e[k + 3] = 1.0
        assert abs(op(e, H) * den * H ** p - w[k + 3]) < TOL, (name, k)


def test_point_mixed_weights():
    den, m = G["dmix"]
    for ia in range(-3, 4):
        for ib in range(-3, 4):
            e = np.zeros((7, 7))
            e[ia + 3, ib + 3] = 1.0
            got = fd.dmix_point(e, H, 2 * H) * den * H * (2 * H)
            k = abs(ia)
            want = 0.0
            if k and abs(ib) == k:
                want = m[k - 1] * (1.0 if ia == ib else -1.0)
            assert abs(got - want) < TOL, (ia, ib, got, want)


SHAPE = (8, 10, 12)  # (nz, ny, nx)
HS = (0.5, 0.25, 2.0)  # spacing along x, y, z: unequal and not 1


def _grid():
    nz, ny, nx = SHAPE
    return fd.Grid(nx, ny, nz, nx * HS[0], ny * HS[1], nz * HS[2])


def _impulse():
    f = np.zeros(SHAPE)
    f[0, 0, 0] = 1.0
    return f


@pytest.mark.parametrize("name, op", [("d1", fd.grid_d1), ("d2", fd.grid_d2)])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_grid_operator_weights(name, op, axis):
    """Operator at point i of an impulse at 0: sum_k w_k delta(i + k) = w_{-i}."""
    den, w = G[name]
    out = op(_impulse(), _grid(), axis) * den * HS[axis] ** (1 if name == "d1" else 2)
    n = SHAPE[2 - axis]
    want = np.zeros(SHAPE)
    for i in range(-3, 4):
        idx = [0, 0, 0]
        idx[2 - axis] = i % n
        want[tuple(idx)] = w[-i + 3]
    assert np.abs(out - want).max() < TOL


@pytest.mark.parametrize("a, b", [(0, 1), (0, 2), (1, 2)])
def test_grid_mixed_weights(a, b):
    """D_ab of an impulse at 0 at point (i_a, i_b): +m_k where i_a = i_b = +-k,
    -m_k where i_a = -i_b = +-k, nothing elsewhere."""
    den, m = G["dmix"]
    out = fd.grid_dmix(_impulse(), _grid(), a, b) * den * HS[a] * HS[b]
    want = np.zeros(SHAPE)
    for k in range(1, 4):
        for sa in (1, -1):
            for sb in (1, -1):
                idx = [0, 0, 0]
                idx[2 - a] = (sa * k) % SHAPE[2 - a]
                idx[2 - b] = (sb * k) % SHAPE[2 - b]
                want[tuple(idx)] = m[k - 1] * (1.0 if sa == sb else -1.0)
    assert np.abs(out - want).max() < TOL


# Planted mistakes in a CPU copy of the oracle that the golden weights must
# reject: the stencil mutants of the mutant suite, a weight typo, and a
# flipped sampling direction of the grid operators (which leaves the point
# stencils right and mirrors every grid derivative).
GOLDEN_MUTANTS = {
    "d1_weight_typo": ("(-s[0] + 9.0 * s[1]", "(-s[0] + 8.0 * s[1]"),
    "gather_direction": ("q[axis] += m;", "q[axis] -= m;"),
}


def _golden_checks():
    checks = [lambda n=n, op=op: test_point_stencil_weights(n, op)
              for n, op in (("d1", fd.d1_point), ("d2", fd.d2_point))]
    checks.append(test_point_mixed_weights)
    checks += [lambda n=n, op=op, a=a: test_grid_operator_weights(n, op, a)
               for n, op in (("d1", fd.grid_d1), ("d2", fd.grid_d2)) for a in (0, 1, 2)]
    checks += [lambda a=a, b=b: test_grid_mixed_weights(a, b) for a, b in ((0, 1), (0, 2), (1, 2))]
    return checks


@pytest.mark.parametrize("name", ["d1_sign", "d2_h_not_squared", "dmix_k2_sign", "dmix_index",
                                  "d1_weight_typo", "gather_direction"])
def test_golden_weights_reject_planted_mistake(name, tmp_path):
    import test_oracle_mutants as M
    from oracle import build_oracle
    old, new = GOLDEN_MUTANTS.get(name) or M.MUTANTS[name]
    so = M._build_mutant(str(tmp_path), name, old, new)
    saved = fd._lib
    try:
        fd._lib = None
        real_build = build_oracle.build
        build_oracle.build = lambda force=False: so
        try:
            fd.lib()
        finally:
            build_oracle.build = real_build
        failures = 0
        for check in _golden_checks():
            try:
                check()
            except AssertionError:
                failures += 1
        assert failures > 0, f"mutant {name} matched every printed weight"
    finally:
        fd._lib = saved
