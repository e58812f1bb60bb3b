"""Kernel variants that split a node's work over more threads give the same
bits as the plain kernels: the volume stage's k_volume_split (knob
DG_VOLUME_SPLIT, 2 = on every level, 0 = off) and the two-warp flux pass of
conforming levels, k_mortar_conf_flux (DG_MORTAR_FLUX_SPLIT, 2 = on every
level, 0 = off).  Child processes evaluate the same residuals and V-cycles with each
setting: plate with every boundary type, 3D mortars, curved shell (random
orders), and uniform-order plate, rotated box (all face orientations) and
curved shell (conforming mortars), in FP64, double-float and the tangent
arithmetic."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
import __graft_entry__ as g
g.build()
from paper_1806_11456_gb300 import dg, synthetic as syn
out = {}
plate = syn.box_mesh(np.linspace(-0.2, 1, 6), [0, 0.01, 0.05, 0.12, 0.3],
                     bc=dict(xmin=1, xmax=2, ymin=lambda i, k: 3 if i < 1 else 4, ymax=1))
rot = syn.rotate_elements(syn.periodic_box(2, 2, 2), seed=4, frac=0.75)
shell = syn.rotate_elements(syn.cubed_sphere_mesh(2, 2), seed=5, frac=0.6)
cases = {
    "plate": (plate, syn.random_orders(plate["K"], 2, 1, 5, 13), syn.flow_params(mach=0.2, re=1e4)),
    "mortars3d": (syn.periodic_box(3, 2, 2), None, syn.flow_params(mach=0.3, re=100.0)),
    "sphere": (shell, None, syn.flow_params(mach=0.2, re=200.0)),
    "plate_uniform": (plate, syn.uniform_orders(plate["K"], 2, 4), syn.flow_params(mach=0.2, re=1e4)),
    "rotated_uniform": (rot, syn.uniform_orders(rot["K"], 3, 3), syn.flow_params(mach=0.3, re=50.0)),
    "sphere_uniform": (shell, syn.uniform_orders(shell["K"], 3, 4), syn.flow_params(mach=0.2, re=200.0)),
}
for name, (mesh, o, prm) in cases.items():
    if o is None:
        o = syn.random_orders(mesh["K"], 3, 1, 4, 14)
    q = torch.tensor(syn.oblique_state(mesh, o, prm, 3), device="cuda")
    for arith in ("fp64", "df32", "mixed"):
        M = dg.Mesh(mesh, o, prm).set_arithmetic(arith)
        if arith == "mixed":
            out[f"{name}_{arith}_tangent"] = M.residual_tangent(q, q * 1e-3).cpu().numpy()
        else:
            out[f"{name}_{arith}_residual"] = M.residual(q).cpu().numpy()
        qc = q.clone()
        M.vcycle(qc, None, beta1=1, beta2=1, beta_c=2, graph=True)
        out[f"{name}_{arith}_vcycle"] = qc.cpu().numpy()
np.savez(OUT, **out)
'''


def _run(tmp_path, **knobs):
    tag = "_".join(f"{k}{v}" for k, v in sorted(knobs.items()))
    path = str(tmp_path / f"split_{tag}.npz")
    env = dict(os.environ, **{k: str(v) for k, v in knobs.items()})
    code = CHILD.replace("ROOT", repr(ROOT)).replace("OUT", repr(path))
    subprocess.run([sys.executable, "-c", code], env=env, check=True, cwd=ROOT)
    return dict(np.load(path))


@pytest.mark.parametrize("knob,off,on", [("DG_VOLUME_SPLIT", 0, 2), ("DG_MORTAR_FLUX_SPLIT", 0, 2)])
def test_split_kernels_give_the_same_bits(tmp_path, knob, off, on):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    a = _run(tmp_path, **{knob: off})
    b = _run(tmp_path, **{knob: on})
    assert set(a) == set(b) and len(a) == 36
    for k in a:
        assert np.array_equal(a[k], b[k], equal_nan=True), k
