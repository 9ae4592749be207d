"""Build the FP64 CPU oracle (test infrastructure) as a shared library.

The oracle is plain C99 compiled with -ffp-contract=off so that it rounds
identically on x86-64 and aarch64 (no fused multiply-add contraction).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lor_oracle.c")
LIB = os.path.join(HERE, "liblor_oracle.so")


def build_oracle(force: bool = False) -> str:
    """Compile oracle/lor_oracle.c into oracle/liblor_oracle.so if stale."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
