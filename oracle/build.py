"""Compiles the CPU oracle (oracle.c) into oracle/_build/liboracle.so.

-ffp-contract=off keeps every FP64 multiply and add separately rounded (GCC
would otherwise fuse them into FMAs on Arm hosts).
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def lib_path(variant: str = "") -> str:
    return os.path.join(HERE, "_build", f"liboracle{variant}.so")


def build(defines=(), variant: str = "", quiet: bool = True) -> str:
    """Build the oracle; `defines`/`variant` let tests build planted-mistake copies."""
    out = lib_path(variant)
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", "-D_GNU_SOURCE", *[f"-D{d}" for d in defines],
           os.path.join(HERE, "oracle.c"), "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True, capture_output=quiet)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(quiet=False))
