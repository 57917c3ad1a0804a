"""Shared test helpers (no method arithmetic)."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def site_err(got, ref):
    """max over sites of |got(x) - ref(x)|_2 / max(|ref(x)|_2, rms_x |ref|_2)."""
    g = np.asarray(got).reshape(-1, 12)
    r = np.asarray(ref).reshape(-1, 12)
    d = np.linalg.norm(g - r, axis=1)
    n = np.linalg.norm(r, axis=1)
    rms = np.sqrt(np.mean(n ** 2))
    return float(np.max(d / np.maximum(n, rms)))


def header_functions():
    """Function names declared in include/dw.h."""
    txt = open(os.path.join(ROOT, "include", "dw.h")).read()
    return sorted(set(re.findall(r"^(?:dw_status|const char\*)\s+(dw_\w+)\s*\(", txt, re.M)))


def parity_of_sites(dims):
    V = int(np.prod(dims))
    s = np.arange(V)
    x = s % dims[0]
    y = (s // dims[0]) % dims[1]
    z = (s // (dims[0] * dims[1])) % dims[2]
    t = s // (dims[0] * dims[1] * dims[2])
    return (x + y + z + t) % 2
