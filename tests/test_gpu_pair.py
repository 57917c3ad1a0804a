"""The 16-bit stencil with two right-hand sides per thread (each link loaded,
and its third row rebuilt, once for both), selected through the tuning file
(DW_TUNE_CACHE) in a fresh process: its outputs must be bitwise equal to the
one-right-hand-side stencil's (dw_apply_noalloc, the same per-site arithmetic
in the same order), match the oracle, and a 12-source solve run with it must
certify to 1e-10."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, os, sys
import numpy as np
sys.path.insert(0, os.environ["REPO"])
sys.path.insert(0, os.path.join(os.environ["REPO"], "tests"))
import torch
torch.cuda.set_device(0)
from helpers import parity_of_sites, site_err
from oracle import oracle as O
from paper_2001_05218_gb300 import dw, inputs as I
dims, kappa, n = (6, 10, 6, 6), 0.122, 12
out = {}
par = parity_of_sites(dims)
U = I.gauge_field(dims, "exp", 91, 1, 0.5)
psis = np.stack([I.gaussian_spinor(dims, 91, 10 + r) for r in range(n)])
for prec, c12 in (("f16", 1), ("bf16", 0)):
    P = dw.PREC[prec]
    Ug = dw.gauge(dims, kappa, U, prec=P, compress12=c12)
    for kind in ("full", "even"):
        if kind == "full":
            src, k, keep = psis, dw.DW_SPINOR_FULL, np.ones(len(par), dtype=bool)
        else:
            keep = par == 0
            src, k = np.where(keep[None, :, None, None], psis, 0), dw.DW_SPINOR_EVEN
        x = dw.spinor(dims, src[:, keep], kind=k, prec=P, nrhs=n)
        a = dw.spinor(dims, kind=k, prec=P, nrhs=n)
        b = dw.spinor(dims, kind=k, prec=P, nrhs=n)
        for dag in (0, 1):
            dw.apply(Ug, x, a, dag=bool(dag))
            dw.check(dw.dw_apply_noalloc(Ug.handle, x.handle, b.handle, dag, dw.current_stream()))
            ga, gb = a.download(), b.download()
            err = 0.0
            for r in range(n):
                ref = O.dirac(dims, kappa, U, src[r], dag=bool(dag)) if kind == "full" else \
                    O.schur(dims, kappa, U, src[r], parity=0, dag=bool(dag))[keep]
                err = max(err, site_err(ga[r], ref))
            out["%s_%s_%d" % (prec, kind, dag)] = {"bitwise": bool(np.array_equal(ga, gb)), "err": err}
Ug = dw.gauge(dims, kappa, U)
bg, xg = dw.spinor(dims, psis, nrhs=n), dw.spinor(dims, nrhs=n)
s, st = dw.cg_solve(Ug, bg, xg, dw.params(tol=1e-10, inner="f16", compress12=1, outer="df64"))
xs = xg.download()
out["solve_status"] = int(s)
out["solve_resid"] = max(float(np.linalg.norm(O.dirac(dims, kappa, U, xs[r]) - psis[r]) / np.linalg.norm(psis[r]))
                         for r in range(n))
print(json.dumps(out))
'''


def test_pair_stencil_selected_by_tuning_file(tmp_path):
    import torch
    assert torch.cuda.is_available()
    dev = torch.cuda.get_device_name(0).replace(" ", "_")
    dims = "6x10x6x6"
    lines = []
    for prec in ("f16c12", "bf16c18"):  # dw_apply keys, T = 32, two thread groups of two RHS
        lines.append("%s/v5/%s/r12/%s 32 2 1" % (dev, prec, dims))
    # the solver's key for its FP16 12-real inner stencil
    cache = tmp_path / "tune.txt"
    cache.write_text("\n".join(lines) + "\n")
    env = dict(os.environ, DW_TUNE_CACHE=str(cache), REPO=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    for key, v in res.items():
        if key.startswith("solve"):
            continue
        tol = 4e-3 if key.startswith("f16") else 3e-2
        assert v["bitwise"], key
        assert v["err"] <= tol, (key, v)
    assert res["solve_status"] == 0 and res["solve_resid"] <= 1e-10
