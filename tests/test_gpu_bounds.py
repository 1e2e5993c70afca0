"""The bounds-checked build (FLB_BOUNDS_CHECK, libflb_check.so) over the
shapes, launch paths, patterns and formats the parity tests use: every global
access of the stream-collide kernels checks its span against the buffer it
addresses, so an index outside would be counted (and not made) instead of
faulting.  The guard itself is exercised by flb_bounds_selftest, which makes
it check two spans just outside a buffer without touching memory."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKLOAD = r'''
import json
import numpy as np
from paper_0707_1581_gb300 import flb
assert flb.LIB_PATH.endswith("libflb_check.so"), flb.LIB_PATH
cases = []

def run(cfgs, steps, host_step=False):
    ctx = flb.flb_create_batch(cfgs) if len(cfgs) > 1 else flb.flb_create_ex(cfgs[0])
    with ctx:
        ctx.flb_step(steps)
        if host_step:
            host = np.zeros(ctx.flb_state_bytes(), np.uint8)
            ctx.flb_state_download(host)
            ctx.flb_step_host(host, 2)
        cases.append([[c.nx, c.ny, c.nz, c.store, c.pattern, c.sites_per_thread, c.block_x, c.block_y, c.lattice]
                      for c in cfgs[:1]] + [ctx.flb_bounds_violations()])

d3 = [(1, 1, 1), (2, 2, 2), (3, 4, 5), (7, 5, 3), (33, 2, 3), (13, 6, 5), (16, 8, 8), (64, 16, 6)]
launches = [((13, 6, 5), 1, 32, 4), ((12, 6, 5), 2, 32, 4), ((12, 6, 5), 4, 4, 8), ((12, 6, 5), 4, 32, 1),
            ((24, 5, 3), 2, 4, 8), ((256, 3, 3), 2, 32, 2), ((512, 2, 2), 4, 128, 1), ((128, 3, 5), 4, 32, 2),
            ((256, 5, 3), 4, 64, 2), ((64, 5, 3), 4, 16, 4), ((8, 7, 3), 4, 2, 16), ((4, 9, 2), 4, 1, 32),
            ((32, 6, 4), 2, 16, 2)]
for pattern in ("ab", "aa"):
    for store in ("f32", "f16dev", "f64", "bf16sr"):
        for shape in d3:
            run([flb.config(*shape, 1.0, 1e-4, 0.3, 0.2, 0.1, 3, store=store, pattern=pattern, force_amp=1e-5)], 3)
    for shape, V, bx, by in launches:
        run([flb.config(*shape, 1.0, 1e-4, 0.3, 0.2, 0.1, 3, store="f32", pattern=pattern, sites_per_thread=V,
                        block_x=bx, block_y=by)], 3)
        run([flb.config(*shape, 1.0, 1e-4, 0.3, 0.2, 0.1, 3, store="f16dev", pattern=pattern, sites_per_thread=V,
                        block_x=bx, block_y=by)], 3)
    for V in (0, 2, 4):
        shapes = [(8, 8, 8), (12, 6, 5), (32, 16, 4), (64, 3, 7), (5, 3, 7)]
        run([flb.config(*sh, 1.0, 1e-4, 0.3, 0.2, 0.0, 3, replica=r, store="f32", pattern=pattern,
                        sites_per_thread=V if sh[0] % 4 == 0 else 0) for r, sh in enumerate(shapes)], 3)
    for shape in ((1, 1), (3, 2), (37, 23), (130, 5), (64, 24), (16, 12)):
        for store in ("f32", "f64", "f16dev"):
            run([flb.config(shape[0], shape[1], 1, 1.0, 1e-4, 0.3, 0.2, 0.1, 3, store=store, pattern=pattern,
                            force_amp=1e-5, lattice="d2q9")], 3)
    run([flb.config(64, 16, 40, 1.0, 1e-4, 0.3, 0.2, 0.0, 3, store="f32", pattern=pattern)], 1, host_step=True)
with flb.flb_create_ex(flb.config(16, 8, 8, store="f32")) as ctx:
    ctx.flb_bounds_selftest()
    selftest = ctx.flb_bounds_violations()
print(json.dumps({"cases": len(cases), "violations": sum(c[-1] for c in cases),
                  "bad": [c for c in cases if c[-1]], "selftest": selftest}))
'''


def test_bounds_checked_build_reports_no_violation():
    from paper_0707_1581_gb300 import build as B
    B.build(check=True)
    env = dict(os.environ, FLB_LIBRARY="check")
    out = subprocess.run([sys.executable, "-c", WORKLOAD], env=env, capture_output=True, text=True, cwd=ROOT,
                         timeout=900)
    assert out.returncode == 0, out.stderr[-3000:]
    res = json.loads(out.stdout.strip().splitlines()[-1])
    assert res["selftest"] == 2                 # the guard counts spans outside the buffer
    assert res["cases"] == 160
    assert res["violations"] == 0, res["bad"]
