"""The bounds-checked build (libairgb_check.so, -DAL_CHECK=1) on the GPU: in
a fresh process that loads it, the fused and step objectives (MSE, NCC, LCC;
2D and 3D), the warp and the learned initialisation's layers run with every
gather index verified; no index leaves its range (the device error words stay
clear) and the objectives still meet the hot path's bars against the oracle."""
import os
import subprocess
import sys

import pytest
import torch

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np, torch
import oracle
from paper_1806_09907_gb300 import build
build.build(checked=True)
from paper_1806_09907_gb300 import airgb, learned_init, synth
assert airgb.LIB_PATH.endswith("libairgb_check.so")
dev = torch.device("cuda", 0)
for shape, delta in (((21, 30, 38), 5), ((24, 40, 52), 6), ((61, 50), 8)):
    F, M = synth.ct_pair(shape, n_inner=6) if len(shape) == 3 else synth.blob_pair(
        shape, 10, (3.0, 8.0), 2.0)
    c = synth.random_ctrl(oracle.lattice_shape(shape, delta), len(shape), 2.0, 9907)
    for sim in ("mse", "ncc", "lcc"):
        pr = airgb.make_problem(shape, delta, sim, 0.1, 1e-5, 7)
        ref, gref = oracle.objective_grad(airgb.SIM_KINDS[sim], F, M, c, delta, 0.1, 1e-5, 7)
        for fused in (True, False):
            val, g = airgb.al_objective_grad(pr, *(torch.from_numpy(a).to(dev) for a in (F, M, c)),
                                             fused=fused)
            val, g = val.cpu().numpy(), g.cpu().numpy()
            assert abs(val[0] - ref["J"]) <= 1e-5 * abs(ref["J"]), (shape, sim, fused)
            assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref), (shape, sim, fused)
res = learned_init.train(learned_init.InitNet((40, 33, 48), 2, dev, seed=3), pairs=6)
assert np.all(np.isfinite(res.losses))
st = airgb.al_get_device_error()
assert st == 0, st
print("checked build clean")
"""


def test_checked_build_runs_clean():
    env = dict(os.environ, AIRGB_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked build clean" in r.stdout
