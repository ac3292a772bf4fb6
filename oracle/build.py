"""Builds the C oracle into a shared library beside its source.

Test infrastructure: ``__graft_entry__.build()`` calls this so the checker
exists on every machine, and the oracle package calls it lazily.  Variants
with ``plant > 0`` are deliberately wrong builds used only by the tests that
check that the pins catch such mistakes.
"""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "domagg_oracle.c")


def library_path(plant: int = 0) -> str:
    name = "libdomagg_oracle.so" if plant == 0 else f"libdomagg_oracle_plant{plant}.so"
    return os.path.join(_HERE, name)


def build_oracle(plant: int = 0, force: bool = False) -> str:
    out = library_path(plant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    tmp = f"{out}.{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", f"-DORACLE_PLANT={plant}",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_oracle(force=True))
