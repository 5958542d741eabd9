"""Build the CPU oracle (test infrastructure) into oracle/libpw_oracle.so.

Plain gcc, no vectorisation flags, no FMA contraction (-ffp-contract=off) so the
single-precision variant evaluates the expression order written in the source.
Builds on x86_64 and aarch64 alike (no target-specific flags).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libpw_oracle.so")
SRC = [os.path.join(HERE, "pw_oracle.c")]
DEPS = SRC + [os.path.join(HERE, "pw_oracle_body.h")]


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB):
        lib_m = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= lib_m for d in DEPS):
            return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", LIB + ".tmp"] + SRC + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
