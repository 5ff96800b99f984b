"""Reader of the hand-worked fixtures under tests/golden/ (no method arithmetic).

A fixture is plain text: '#' comments carry the derivation and the passages of
the paper it follows; every other line is `key = value` with a Python literal
value. `let name = "expr"` defines a named closed form. Real values are
closed-form expressions in p = fp32(0.6), q = fp32(0.8), the names defined by
`let`, + - * / **, and sqrt(); they are evaluated in FP64 by a small
whitelisting evaluator (no eval()).
"""
from __future__ import annotations

import ast
import math
import operator
import os

import numpy as np

from synth.corpus import Corpus, from_dense

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FIXTURES = sorted(f[:-4] for f in os.listdir(GOLDEN_DIR) if f.endswith(".txt"))

_BINOPS = {ast.Add: operator.add, ast.Sub: operator.sub, ast.Mult: operator.mul,
           ast.Div: operator.truediv, ast.Pow: operator.pow}


def _evaluate(expr: str, env: dict) -> float:
    def ev(n):
        if isinstance(n, ast.Expression):
            return ev(n.body)
        if isinstance(n, ast.Constant) and isinstance(n.value, (int, float)) and not isinstance(n.value, bool):
            return float(n.value)
        if isinstance(n, ast.Name) and n.id in env:
            return env[n.id]
        if isinstance(n, ast.BinOp) and type(n.op) in _BINOPS:
            return _BINOPS[type(n.op)](ev(n.left), ev(n.right))
        if isinstance(n, ast.UnaryOp) and isinstance(n.op, ast.USub):
            return -ev(n.operand)
        if (isinstance(n, ast.Call) and isinstance(n.func, ast.Name) and n.func.id == "sqrt"
                and len(n.args) == 1 and not n.keywords):
            return math.sqrt(ev(n.args[0]))
        raise ValueError(f"unsupported expression element {ast.dump(n)} in {expr!r}")
    return ev(ast.parse(expr, mode="eval"))


class Golden:
    """One parsed fixture: g["r1.labels"], g.num("u1.objective"), g.nums(...)."""

    def __init__(self, name: str):
        self.name = name
        self._kv: dict = {}
        self._env = {"p": float(np.float32(0.6)), "q": float(np.float32(0.8))}
        with open(os.path.join(GOLDEN_DIR, name + ".txt")) as f:
            for ln, line in enumerate(f, 1):
                s = line.strip()
                if not s or s.startswith("#"):
                    continue
                key, sep, val = s.partition("=")
                if not sep:
                    raise ValueError(f"{name}:{ln}: expected 'key = value'")
                key, v = key.strip(), ast.literal_eval(val.strip())
                if key.startswith("let "):
                    self._env[key[4:].strip()] = _evaluate(v, self._env)
                else:
                    self._kv[key] = v
        self.D, self.k = int(self["D"]), int(self["k"])
        self.iterations = int(self["iterations"])
        self.modes = list(self["modes"])
        self.seeds = np.asarray(self["seeds"], dtype=np.int32)

    def __getitem__(self, key):
        return self._kv[key]

    def __contains__(self, key):
        return key in self._kv

    def num(self, key) -> float:
        return _evaluate(self._kv[key], self._env)

    def nums(self, key) -> np.ndarray:
        v = self._kv[key]
        if v and isinstance(v[0], list):
            return np.array([[_evaluate(e, self._env) for e in row] for row in v], dtype=np.float64)
        return np.array([_evaluate(e, self._env) for e in v], dtype=np.float64)

    def dense(self) -> np.ndarray:
        """The documents as a dense fp32 matrix (each value exactly 1, p or q)."""
        docs = self["docs"]
        X = np.zeros((len(docs), self.D), dtype=np.float32)
        for i, row in enumerate(docs):
            for t, e in row:
                x = _evaluate(e, self._env)
                assert float(np.float32(x)) == x, "document values must be fp32 numbers"
                X[i, t] = x
        return X

    def corpus(self) -> Corpus:
        return from_dense(self.dense())
