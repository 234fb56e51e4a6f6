"""Writes tests/golden/raster_work_<workload>.json: the oracle's count of
front-facing triangles reaching the image and of covered fragments per
rendered view, averaged over a sample of the workload's environments and
steps.  These are properties of the workload, not of any kernel; the bench
takes them as the algorithmic work of the rasteriser for its roofline.

    python -m oracle.raster_work apartments4096
"""
import json
import os
import sys

import numpy as np

import oracle as O
from paper_2306_07552_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def measure(name, n_envs=32, n_steps=8):
    w = I.WORKLOADS[name]
    scenes = I.make_scenes(w)
    robot = I.fetch_like_robot()
    env_scene = I.env_scene_map(w.n_envs, w.n_scenes)
    envs = [int(e) for e in np.linspace(0, w.n_envs - 1, n_envs)]
    acts = I.make_actions(n_steps, len(envs), w.action_dist, seed=w.action_seed)
    tri, frag, amb = [], [], []
    orcs = {}
    for i, e in enumerate(envs):
        s = int(env_scene[e])
        if s not in orcs:
            mesh = I.unit_cube() if w.objects == "boxes" else I.icosahedron()
            orcs[s] = O.Oracle(robot, scenes[s], mesh, I.object_colors(64))
        st = O.Oracle.make_state((0, 0, 0), np.zeros(7))
        st.boxes = 1 if w.objects == "boxes" else 0
        orcs[s].reset(st, w.reset_seed, e, w.n_objects, *w.obj_radius)
        for t in range(n_steps):
            orcs[s].step(st, acts[t, i])
            _, _, a, _, stats = orcs[s].render(st, w.img, w.img)
            tri.append(stats.tris_setup)
            frag.append(stats.frags_covered)
            amb.append(float(a.mean()))
    return {"workload": name, "views": len(tri), "tris_per_view": float(np.mean(tri)),
            "frags_per_view": float(np.mean(frag)), "tris_per_view_max": int(np.max(tri)),
            "frags_per_view_max": int(np.max(frag)), "ambiguous_frac": float(np.mean(amb)),
            "sample": f"{len(envs)} envs x {n_steps} steps from reset, oracle trajectories"}


if __name__ == "__main__":
    for name in (sys.argv[1:] or ["apartments4096"]):
        d = measure(name)
        p = os.path.join(ROOT, "tests", "golden", f"raster_work_{name}.json")
        json.dump(d, open(p, "w"), indent=1)
        print(p, d)
