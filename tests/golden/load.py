"""Reader for the small text fixtures in this folder (name = python expression)."""
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def load(name):
    out = {}
    with open(os.path.join(HERE, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, expr = (x.strip() for x in line.split("=", 1))
            out[key] = expr
    return out


def evaluate(expr, **env):
    scope = {"sqrt": math.sqrt, "exp": math.exp}
    scope.update(env)
    return eval(expr, {"__builtins__": {}}, scope)
