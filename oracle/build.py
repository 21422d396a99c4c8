"""Build the FP64 CPU oracle (``liboracle.so``) with the system C compiler.

Test infrastructure: the oracle is compiled so that tests and the CPU
baseline can run it; the product library never links it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "opo_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

# IEEE FP64 throughout: no fast-math and no FMA contraction, so the oracle's
# rounding is the textbook one on any host (x86_64 here, aarch64 on the GPU machine).
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-Wall", "-Wextra"]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source if missing or stale.

    ``OPO_ORACLE_LIB`` names a prebuilt oracle library to load instead (the
    mutation test uses it to load deliberately broken copies)."""
    override = os.environ.get("OPO_ORACLE_LIB")
    if override:
        return override
    hdr = os.path.join(HERE, "opo_oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return LIB
    cc = os.environ.get("CC", "gcc")
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call([cc, *CFLAGS, "-o", tmp, SRC, "-lm"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
