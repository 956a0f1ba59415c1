"""Compile the C part of the oracle (``quant.c``) into ``_quant.so`` with gcc.

Plain portable C11 + ``unsigned __int128`` (gcc on x86_64 and aarch64); no
architecture flags, so the same source builds on x86 and Arm.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "quant.c")
LIB = os.path.join(HERE, "_quant.so")


def build_oracle(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-Wall", "-o", tmp, SRC, "-lm"])
    os.replace(tmp, LIB)
    return LIB
