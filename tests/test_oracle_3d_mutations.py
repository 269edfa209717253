"""Plant plausible three-dimensional mistakes in the oracle's hierarchy and
in the 3-D inputs (on the CPU) and check that the 3-D pins catch each of
them: the child-slot order, the row-major cell key and the distance between
closed cubes each forgetting the z axis, a wrong trilinear stiffness entry,
and the element matrix without its cell-size factor."""
import inspect
import itertools
import types

import numpy as np
import pytest

import oracle.hierarchy as hier
import workloads.rough3d as r3
from workloads import make_problem3


def _mutated_module(mod, old, new, name):
    src = inspect.getsource(mod)
    assert old in src, name
    m = types.ModuleType(mod.__name__ + "_mut")
    m.__dict__["__package__"] = mod.__package__
    exec(compile(src.replace(old, new), "<mutant>", "exec"), m.__dict__)
    return m


HIER_MUTATIONS = {
    "slot_without_z": ("slot = sum((cells[:, a] & 1) << a for a in range(self.d))",
                       "slot = sum((cells[:, a] & 1) << a for a in range(2))"),
    "key_without_z": ("for a in range(c.shape[1] - 1, -1, -1):\n        key = key * (1 << k) + c[:, a]",
                      "for a in range(1, -1, -1):\n        key = key * (1 << k) + c[:, a]"),
    "distance_without_z": ("dist = np.abs(c - c[i])", "dist = np.abs(c[:, :2] - c[i, :2])"),
}


def _hierarchy_pins(H_cls):
    """The 3-D hierarchy pins of test_oracle_3d.py, on a given Hierarchy
    class; returns True when every one holds."""
    p = make_problem3(8, 10, 1)
    H = H_cls(p.cells, p.q)
    if [H.n(k) for k in range(1, p.q + 1)] != [8, 64, 343]:
        return False
    for k in range(2, p.q + 1):
        P = H.pi(k).toarray()
        W2 = H.W(k, "const2").toarray()
        if W2.shape[0] != H.n(k) - H.n(k - 1) or np.abs(P @ W2.T).max() > 1e-14:
            return False
    c = H.levels[p.q].cells
    for ch in H.children(p.q):
        slot = (c[ch, 0] & 1) + 2 * (c[ch, 1] & 1) + 4 * (c[ch, 2] & 1)
        if not np.all(np.diff(slot) > 0):
            return False
    q = make_problem3(16, 10, 0)
    H = H_cls(q.cells, q.q)
    cc = H.levels[3].cells
    i = int(np.nonzero((cc == 4).all(axis=1))[0][0])
    if len(H.neighbours(3, 1, "euclid")[i]) != 81:
        return False
    return True


def test_hierarchy_pins_hold_unmutated():
    assert _hierarchy_pins(hier.Hierarchy)


@pytest.mark.parametrize("name", sorted(HIER_MUTATIONS))
def test_hierarchy_pins_catch_mutation(name):
    old, new = HIER_MUTATIONS[name]
    m = _mutated_module(hier, old, new, name)
    assert not _hierarchy_pins(m.Hierarchy)


INPUT_MUTATIONS = {
    "edge_diagonal_entry": ("2: -1.0 / 12.0, 3: -1.0 / 12.0", "2: -1.0 / 6.0, 3: -1.0 / 12.0"),
    "no_cell_size_factor": ("av = a.ravel() * h", "av = a.ravel()"),
}


def _input_pins(mod):
    """Quadrature of the trilinear gradients and the energy of a trilinear
    interpolant, against the module's K_REF3 and assembly."""
    t = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    pts = [np.array(x) for x in itertools.product(t, t, t)]

    def grad(c, x):
        b = [(c >> a) & 1 for a in range(3)]
        f = [x[a] if b[a] else 1.0 - x[a] for a in range(3)]
        df = [1.0 if b[a] else -1.0 for a in range(3)]
        return np.array([df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2]])

    K = sum(0.125 * np.array([grad(c, x) for c in range(8)]) @
            np.array([grad(c, x) for c in range(8)]).T for x in pts)
    if np.abs(K - mod.K_REF3).max() > 1e-15:
        return False
    n = 4
    h = 1.0 / n
    rng = np.random.default_rng(5)
    a = np.exp(rng.uniform(-1.0, 1.0, (n, n, n)))
    A = mod.assemble_q1_3d(a)
    u = rng.standard_normal((n - 1) ** 3)
    full = np.zeros((n + 1,) * 3)
    full[1:n, 1:n, 1:n] = u.reshape((n - 1,) * 3)
    energy = 0.0
    for cz, cy, cx in itertools.product(range(n), repeat=3):
        vals = [full[cz + ((c >> 2) & 1), cy + ((c >> 1) & 1), cx + (c & 1)] for c in range(8)]
        for x in pts:
            g = sum(v * grad(c, x) for c, v in enumerate(vals)) / h
            energy += a[cz, cy, cx] * 0.125 * h ** 3 * (g @ g)
    return abs(u @ (A @ u) - energy) <= 1e-12 * energy


def test_input_pins_hold_unmutated():
    assert _input_pins(r3)


@pytest.mark.parametrize("name", sorted(INPUT_MUTATIONS))
def test_input_pins_catch_mutation(name):
    old, new = INPUT_MUTATIONS[name]
    m = _mutated_module(r3, old, new, name)
    assert not _input_pins(m)
