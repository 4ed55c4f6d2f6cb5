"""Builds the FP64 CPU oracle (test infrastructure only) into oracle/_build/.

The oracle is plain C compiled with ``-ffp-contract=off`` so that every
``a*b + c`` is two IEEE roundings on both x86-64 and aarch64 hosts.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cem_oracle.c")
SRC_CST = os.path.join(HERE, "cst_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libcem_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or stale; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    deps = [SRC, SRC_CST, os.path.join(HERE, "cem_oracle.h"), os.path.join(HERE, "cst_oracle.h")]
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in deps)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared",
           "-o", tmp, SRC, SRC_CST, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
