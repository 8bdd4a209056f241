"""Operation count of one phase cell of the quantum model, from the oracle's
expression of it (qso_qfp_run with qso_rates_c, qso_gaunt and qso_h2 in
qs_oracle.c, i.e. Eq. 6 with the Fokker-Planck closure as read there).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): it supplies the algorithmic
work per unit that the roofline of the phase-integrating kernels is stated
against, and is not part of the product.

The cell is written once, as the oracle evaluates it, over a small expression
graph with common subexpressions merged.  Quantities that depend only on the
sample (a_eff, gamma0) or the laser are loop-invariant and not counted; the
per-cell inputs are the state (du, V, the previous Gaunt factor) and the
envelope G_j of the cell (a table: the envelope is data, not arithmetic, in
every implementation).  Costs, in the units of the GPU's pipes:
  add, sub, mul                 1 FMA-pipe operation each; a product whose only
                                use is one add or sub fuses with it (one FMA)
  division x / y                a reciprocal (MUFU) and a product
  log(x)                        a base-2 logarithm (MUFU) and a product (ln 2)
  x**p, p not an integer        lg2 and ex2 (MUFU) and a product
  x**n, n a small integer       n - 1 products
MUFU work is counted in issue slots of the rcp / lg2 rate: ex2 issues at
twice that rate on this GPU (the unit-rate probe measures both), so an ex2
counts half a slot.
"""
from __future__ import annotations

from dataclasses import dataclass, field


@dataclass(eq=False)
class Node:
    op: str                       # const, inv, var, add, sub, mul, div, log, powf, neg
    args: tuple = ()
    value: float | None = None    # constants
    name: str = ""
    users: list = field(default_factory=list)

    @property
    def invariant(self):
        if self.op in ("const", "inv"):
            return True
        if self.op == "var":
            return False
        return all(a.invariant for a in self.args)

    def operands(self):
        return self.args


class Graph:
    def __init__(self):
        self.table = {}

    def _key(self, op, args, value=None, name=""):
        return (op, tuple(id(a) for a in args), value, name)

    def node(self, op, *args, value=None, name=""):
        k = self._key(op, args, value, name)
        n = self.table.get(k)
        if n is None:
            n = Node(op, args, value, name)
            self.table[k] = n
        return n

    def const(self, v):
        return self.node("const", value=float(v))

    def inv(self, name):
        return self.node("inv", name=name)

    def var(self, name):
        return self.node("var", name=name)


class V:
    """Arithmetic on graph nodes (constants folded where both sides are)."""

    def __init__(self, g: Graph, n: Node):
        self.g, self.n = g, n

    def _w(self, x):
        return x if isinstance(x, V) else V(self.g, self.g.const(x))

    def _bin(self, op, a, b):
        a, b = self._w(a), self._w(b)
        if a.n.op == "const" and b.n.op == "const":
            x, y = a.n.value, b.n.value
            return V(self.g, self.g.const({"add": x + y, "sub": x - y, "mul": x * y, "div": x / y}[op]))
        return V(self.g, self.g.node(op, a.n, b.n))

    def __add__(self, o): return self._bin("add", self, o)
    def __radd__(self, o): return self._bin("add", o, self)
    def __sub__(self, o): return self._bin("sub", self, o)
    def __rsub__(self, o): return self._bin("sub", o, self)
    def __mul__(self, o): return self._bin("mul", self, o)
    def __rmul__(self, o): return self._bin("mul", o, self)
    def __truediv__(self, o): return self._bin("div", self, o)
    def __rtruediv__(self, o): return self._bin("div", o, self)
    def __neg__(self): return self._bin("mul", self, -1.0)

    def log(self):
        return V(self.g, self.g.node("log", self.n))

    def powf(self, p):
        return V(self.g, self.g.node("powf", self.n, value=float(p)))


def oracle_cell(aS_scale: float = 1.0):
    """The oracle's cell j (qso_qfp_run) as a graph; returns (graph, outputs)."""
    g = Graph()
    c = lambda x: V(g, g.const(x))                     # noqa: E731
    du, Vv, gprev, G = (V(g, g.var(n)) for n in ("du", "V", "gprev", "G"))
    aeff, g0, h, Rc, aS = (V(g, g.inv(n)) for n in ("aeff", "gamma0", "h", "Rc", "aS"))
    A = aeff * G
    K = c(2.0 / 3.0) * Rc * A * A
    du_mid = du + c(0.5) * h * K * gprev
    mu = g0 / (c(1.0) + g0 * du_mid)
    # qso_rates_c: chi at the rms field, Gaunt factor and its derivative,
    # second-moment factor, the three rates
    chi = c(2.0) * mu * (A / c(2.0 ** 0.5)) / (aS * c(aS_scale))
    L1 = (c(1.0) + c(1.7) * chi).log()
    B = c(1.0) + c(4.8) * (c(1.0) + chi) * L1 + c(2.44) * chi * chi
    dB = c(4.8) * L1 + c(4.8) * (c(1.0) + chi) * c(1.7) / (c(1.0) + c(1.7) * chi) + c(2.0 * 2.44) * chi
    gv = B.powf(-2.0 / 3.0)
    gp = c(-2.0 / 3.0) * gv / B * dB
    num = c(1.0) + chi * (c(4.26) + c(0.494) * chi)
    den = c(1.0) + chi * (c(12.32) + chi * (c(17.44) + c(1.63) * chi))
    h2 = gv * num / den
    sf = c(2.0) * gv + chi * gp
    D1 = -(K * mu * mu * gv)
    dD1 = -(K * mu * sf)
    D2 = c(55.0 / (16.0 * 3.0 ** 0.5)) * K * mu * mu * mu * chi * h2
    # the update (the Gaunt factor of the cell is D1 / (-K mu^2) = g)
    lam = c(2.0) * dD1
    rv = lam * Vv + D2
    du_new = du + h * K * gv
    V_new = Vv + h * rv + c(0.5) * h * h * lam * rv
    return g, [du_new.n, V_new.n, gv.n]


def count(outputs) -> dict:
    """Operations per cell reachable from the outputs, with the fusion and
    MUFU rules of the module docstring."""
    seen, order = set(), []

    def walk(n):
        if id(n) in seen:
            return
        seen.add(id(n))
        for a in n.operands():
            walk(a)
        order.append(n)

    for o in outputs:
        walk(o)
    work = [n for n in order if n.op not in ("const", "inv", "var") and not n.invariant]
    users = {id(n): 0 for n in order}
    for n in order:
        for a in n.operands():
            users[id(a)] += 1
    adds = sum(1 for n in work if n.op in ("add", "sub"))
    muls = 0
    mufu = 0.0
    for n in work:
        if n.op == "mul":
            # a product by -1 or 1 is a sign flip folded into its user
            if not any(a.op == "const" and abs(a.value) == 1.0 for a in n.args):
                muls += 1
        elif n.op == "div":
            # x / y: a reciprocal of y, then a product (a reciprocal alone if
            # x is the constant 1); y invariant: a product by its inverse
            if n.args[1].invariant:
                muls += 1
            else:
                mufu += 1.0
                if not (n.args[0].op == "const" and n.args[0].value == 1.0):
                    muls += 1
        elif n.op == "log":
            mufu += 1.0
            muls += 1
        elif n.op == "powf":
            mufu += 1.5
            muls += 1
    # fusion: each add or sub absorbs one single-use product that costs at
    # least one multiplication
    fused = 0
    for n in work:
        if n.op in ("add", "sub"):
            if any(a.op == "mul" and not a.invariant and users[id(a)] == 1 and
                   not any(b.op == "const" and abs(b.value) == 1.0 for b in a.args)
                   for a in n.args):
                fused += 1
    return {"adds": adds, "muls": muls, "fused": fused, "fma_pipe": adds + muls - fused,
            "mufu_slots": mufu}


def cell_counts() -> dict:
    """Algorithmic work of one phase cell of the quantum model (per sample)."""
    _, outs = oracle_cell()
    return count(outs)


if __name__ == "__main__":
    print(cell_counts())
