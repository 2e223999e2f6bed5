"""Compile the C part of the FP64 oracle (test infrastructure only).

gcc, -O2, -ffp-contract=off so that no multiply-add is fused: the coordinate
rounding of the oracle follows a fixed FP64 operation order.  build(sanitize=
True) makes a second copy instrumented with AddressSanitizer and
UndefinedBehaviorSanitizer (errors fatal), loaded instead of the plain one when
AW_ORACLE_SANITIZE=1 (the process must preload the sanitizer runtimes).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "aw_oracle.c")
LIB = os.path.join(HERE, "_aw_oracle.so")
LIB_SAN = os.path.join(HERE, "_aw_oracle_san.so")
SAN_FLAGS = ["-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer"]


def build(force: bool = False, sanitize: bool = False) -> str:
    lib = LIB_SAN if sanitize else LIB
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= os.path.getmtime(SRC)):
        return lib
    tmp = lib + ".tmp%d" % os.getpid()
    opt = SAN_FLAGS if sanitize else ["-O2"]
    cmd = ["gcc"] + opt + ["-std=c99", "-ffp-contract=off", "-fno-fast-math",
                           "-shared", "-fPIC", SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True))
