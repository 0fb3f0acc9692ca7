"""Build the FP64 CPU oracle into oracle/liboracle.so (test infrastructure).

Plain gcc, no FMA contraction: every product and sum in the oracle is rounded
on its own in the order its source fixes.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "qe_oracle.c")
HDR = os.path.join(HERE, "qe_oracle.h")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR), os.path.getmtime(__file__))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wextra", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def build_variant(source: str, out_path: str) -> str:
    """Compile `source` (a modified copy of qe_oracle.c) with the oracle's own
    flags into out_path; its #include of qe_oracle.h resolves to this folder."""
    src = os.path.splitext(out_path)[0] + ".c"
    with open(src, "w") as f:
        f.write(source)
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-I" + HERE, "-o", out_path, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
