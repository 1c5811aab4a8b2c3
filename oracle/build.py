"""Compile the oracle's plain C helpers (test infrastructure only)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def build() -> str:
    src = os.path.join(HERE, "csrc", "oracle_sketch.c")
    out = os.path.join(HERE, "_oracle_sketch.so")
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", out, src, "-lm"])
    return out


if __name__ == "__main__":
    print(build())
