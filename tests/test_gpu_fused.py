"""The fused smoothing kernel (k_smooth_block: a smoothing block of a small
conforming level in one cooperative launch, its stages separated by grid
barriers; off by default, DG_FUSED_SMOOTH selects it) gives the same bits as
the separate launches.  Child processes run
the same smoothing, V-cycles (direct and graph-replayed, fixed counts and
the residual-based smoothing control of Sec. 3.1.2), batched cycles with a
held solve, and mixed-precision cycles with DG_FUSED_SMOOTH=0 (never fused)
and 2 (every level that qualifies): 2D plate with every boundary type, a
rotated 3D box (all face orientations), a curved shell, a serving-sized
periodic box, and random orders (non-conforming levels above the coarse
ones, which the fused kernel skips)."""
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
box = syn.periodic_box(3, 3, 3)
cases = {
    "plate_uniform": (plate, syn.uniform_orders(plate["K"], 2, 4), syn.flow_params(mach=0.2, re=1e4)),
    "rotated_uniform": (rot, syn.uniform_orders(rot["K"], 3, 3), syn.flow_params(mach=0.3, re=50.0)),
    "sphere_uniform": (shell, syn.uniform_orders(shell["K"], 3, 3), syn.flow_params(mach=0.2, re=200.0)),
    "box_n2": (box, syn.uniform_orders(box["K"], 3, 2), syn.flow_params(mach=0.3, re=100.0)),
    "plate_random": (plate, syn.random_orders(plate["K"], 2, 1, 5, 13), syn.flow_params(mach=0.2, re=1e4)),
}
for name, (mesh, o, prm) in cases.items():
    q0 = syn.oblique_state(mesh, o, prm, 3)
    q = torch.tensor(q0, device="cuda")
    s = torch.tensor(syn.random_source(mesh, o, 5, amp=1e-3), device="cuda")
    for arith in ("fp64", "mixed", "df32"):
        M = dg.Mesh(mesh, o, prm).set_arithmetic(arith)
        qc = q.clone()
        M.smooth(qc, s, sweeps=3)
        out[f"{name}_{arith}_smooth"] = qc.cpu().numpy()
        for graph in (False, True):
            qc = q.clone()
            M.vcycle(qc, s, beta1=2, beta2=1, beta_c=3, graph=graph)
            M.vcycle(qc, s, beta1=2, beta2=1, beta_c=3, graph=graph)
            out[f"{name}_{arith}_vcycle_g{int(graph)}"] = qc.cpu().numpy()
        qc = q.clone()
        rep = M.vcycle(qc, s, beta1=1, beta2=1, beta_c=2, control=4, eta=1.5, want_norm=True)
        out[f"{name}_{arith}_controlled"] = qc.cpu().numpy()
        out[f"{name}_{arith}_controlled_evals"] = np.array([rep["residual_evals"], rep["rnorm"]])
# a batch with a held solve (its time step is masked in every sweep)
items = [(plate, syn.uniform_orders(plate["K"], 2, 3), syn.flow_params(mach=0.2, re=1e4)),
         (plate, syn.uniform_orders(plate["K"], 2, 3), syn.flow_params(mach=0.3, re=1e3)),
         (plate, syn.uniform_orders(plate["K"], 2, 3), syn.flow_params(mach=0.25, re=3e3))]
for arith in ("fp64", "mixed"):
    B = dg.Mesh.batch(items).set_arithmetic(arith)
    qb = torch.tensor(np.concatenate([syn.oblique_state(m, o, p, 7 + k) for k, (m, o, p) in enumerate(items)]),
                      device="cuda")
    B.set_active([1, 0, 1])
    B.vcycle(qb, None, beta1=2, beta2=1, beta_c=3, graph=True)
    B.vcycle(qb, None, beta1=1, beta2=1, beta_c=2, control=4, eta=1.5)
    out[f"batch_held_{arith}"] = qb.cpu().numpy()
np.savez(OUT, **out)
'''


def _run(tmp_path, **knobs):
    tag = "_".join(f"{k}{v}" for k, v in sorted(knobs.items()))
    path = str(tmp_path / f"fused_{tag}.npz")
    env = dict(os.environ, **{k: str(v) for k, v in knobs.items()})
    code = CHILD.replace("ROOT", repr(ROOT)).replace("OUT", repr(path))
    subprocess.run([sys.executable, "-c", code], env=env, check=True, cwd=ROOT)
    return dict(np.load(path))


def test_fused_smoothing_gives_the_same_bits(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    a = _run(tmp_path, DG_FUSED_SMOOTH=0)
    b = _run(tmp_path, DG_FUSED_SMOOTH=2)
    assert set(a) == set(b) and len(a) == 5 * 3 * 5 + 2
    for k in a:
        assert np.array_equal(a[k], b[k], equal_nan=True), k
