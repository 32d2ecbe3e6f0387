"""Test helper: build the in-tree CUDA library once per session if it is
missing or older than its sources."""

import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1409_8116_gb300")


def _stale(lib):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    srcdirs = [os.path.join(PKG, "csrc"), os.path.join(ROOT, "include")]
    for d in srcdirs:
        for f in os.listdir(d):
            if os.path.getmtime(os.path.join(d, f)) > t:
                return True
    return False


def ensure_built():
    lib = os.path.join(PKG, "libpoisfft.so")
    if _stale(lib):
        from paper_1409_8116_gb300 import build
        build.build()
    return lib
