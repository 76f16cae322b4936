"""Helpers for tests of the CUDA library: build once, load, read the header."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def ensure_built():
    from paper_1806_04164_gb300 import LIBPATH
    from paper_1806_04164_gb300.build import build
    srcdir = os.path.join(ROOT, "paper_1806_04164_gb300", "csrc")
    newest = max(os.path.getmtime(os.path.join(srcdir, f)) for f in os.listdir(srcdir))
    newest = max(newest, os.path.getmtime(os.path.join(ROOT, "include", "pie.h")))
    if not os.path.exists(LIBPATH) or os.path.getmtime(LIBPATH) < newest:
        build()
    return LIBPATH


def header_functions():
    text = open(os.path.join(ROOT, "include", "pie.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pie_[a-z_0-9]+)\s*\(", text)))
