"""Helpers comparing the CUDA path (through the C ABI) with the FP64 oracle.

Protocol (lockstep): for every checked environment the oracle starts from the
GPU's FP32 state before the step, widened to FP64, applies the same actions
and must reproduce the GPU's state after the step.  Discrete results (contact
masks, flags, grasp events, held index) must match bit for bit unless the
oracle reports a decision within 1e-4 m of its threshold ("near band"; such
environments are counted and skipped).  Continuous results must agree within
1e-5 m / rad.  Images are rendered by the oracle from the GPU's state after
the step; on pixels the oracle does not flag as ambiguous, coverage and RGB
must match exactly and depth within 1e-5 relative; pixels where the robot's
own body wins get 5e-6 m / |cos| on top (see DEPTH_ABS).
"""
import math

import numpy as np

import oracle as O

POSE_TOL = 1e-5
DEPTH_REL = 1e-5
# Only for pixels whose winner is one of the robot's own spheres: the GPU
# places them by FP32 forward kinematics through the arm's joint chain and
# the oracle by FP64, so a sphere centre differs by up to the lockstep pose
# error (<= 2.5e-6 m); divided by |cos| of the hit (a shift across a slanted
# surface moves the hit along the ray by shift / |cos|) this exceeds 1e-5
# relative at the few-centimetre depths of the robot body.  Every other pixel
# (scene triangles, objects, whose positions both sides read from the same
# state) is held to 1e-5 relative alone.
DEPTH_ABS = 5e-6
# instance slots of the robot's spheres start after the 256 object slots
ROBOT_SLOT0 = 256


def oracle_state(arrs, e, M, boxes=False):
    """The GPU state of environment e widened to FP64 (boxes: the oriented-box
    object model's extents, yaws and carried rotation too)."""
    return O.Oracle.make_state((float(arrs["base_x"][e]), float(arrs["base_z"][e]),
                                float(arrs["yaw"][e])), arrs["q"][:, e], int(arrs["held"][e]),
                               arrs["c_off"][:, e], arrs["p_pre"][:, e], arrs["obj"][e, :M],
                               int(arrs["step"][e]), int(arrs["episode"][e]),
                               task=arrs["task"][e] if "task" in arrs else None,
                               boxes=arrs["box"][e, :M] if boxes else None,
                               r_off=arrs["r_off"][:, e] if boxes else None)


def ang_diff(a, b):
    d = (a - b) % (2 * math.pi)
    return min(d, 2 * math.pi - d)


class Tally:
    def __init__(self):
        self.envs = 0
        self.near_band = 0
        self.events = {}
        self.contacts = 0
        self.pixels = 0
        self.ambiguous = 0
        self.max_pose_err = 0.0
        self.max_depth_rel = 0.0
        self.max_task_err = 0.0        # reward, task observations and task state
        self.near_band_flips = 0       # near-band env-steps whose discrete results differ
        self.robot_pixels = 0          # checked pixels won by the robot's own spheres
        self.fp16_max_err = 0.0        # FP16 depth: largest |gpu - oracle| (m)
        self.fp16_max_frac = 0.0       # ... as a fraction of its bound
        self.per_result = {}           # result name -> largest |gpu - oracle|

    def note(self, name, err):
        err = float(np.max(err)) if np.size(err) else 0.0
        self.per_result[name] = max(self.per_result.get(name, 0.0), err)

    def report(self):
        """One line per result: the largest error seen against the oracle."""
        return "\n".join(f"  {k:<14s} {v:.2e}" for k, v in sorted(self.per_result.items()))

    def __repr__(self):
        r = (f"envs={self.envs} near_band={self.near_band} "
             f"near_band_flips={self.near_band_flips} contacts={self.contacts} "
             f"events={self.events} pixels={self.pixels} ambiguous={self.ambiguous} "
             f"max_pose_err={self.max_pose_err:.2e} max_depth_rel={self.max_depth_rel:.2e} "
             f"max_task_err={self.max_task_err:.2e}")
        if self.fp16_max_frac:
            r += (f" fp16_max_err={self.fp16_max_err:.2e} m "
                  f"fp16_max_of_bound={self.fp16_max_frac:.3f}")
        return r


def check_step(orc, before, after, out, acts, envs, M, tally, step_fn=None, boxes=False):
    """Physics parity of one step for the listed environments.  step_fn(st,
    action, env) replaces the oracle's plain step (e.g. with its neural-SDF
    rule or the paper's heuristics); boxes: the oriented-box object model."""
    mask = out["contact_mask"].cpu().numpy().view(np.uint32)
    flags = out["contact_flags"].cpu().numpy()
    event = out["event"].cpu().numpy()
    held = out["held"].cpu().numpy()
    pose = out["pose"].cpu().numpy()
    objo = out["obj_pos"].cpu().numpy()
    reward = out["reward"].cpu().numpy() if out.get("reward") is not None else None
    tobs = out["task_obs"].cpu().numpy() if out.get("task_obs") is not None else None
    succ = out["success"].cpu().numpy() if out.get("success") is not None else None
    for e in envs:
        st = oracle_state(before, e, M, boxes)
        o = step_fn(st, acts[e], e) if step_fn else orc.step(st, acts[e])
        tally.envs += 1
        same = (mask[e] == o.contact_mask and flags[e] == o.flags and event[e] == o.event
                and held[e] == st.held == after["held"][e])
        if o.near_band:
            # a decision within 1e-4 m of its threshold may go either way in
            # FP32: only the discrete results are excused.  When they agree,
            # everything else is compared as usual; when they differ, the two
            # sides followed different branches and the continuous results
            # have nothing to agree with (counted).
            tally.near_band += 1
            if not same:
                tally.near_band_flips += 1
                continue
        assert mask[e] == o.contact_mask, (e, hex(mask[e]), hex(o.contact_mask))
        assert flags[e] == o.flags, (e, flags[e], o.flags)
        assert event[e] == o.event, (e, event[e], o.event)
        assert held[e] == st.held == after["held"][e], (e, held[e], st.held)
        tally.contacts += int(o.contact_mask != 0)
        tally.events[int(o.event)] = tally.events.get(int(o.event), 0) + 1
        parts = {"base_xz_m": [abs(after["base_x"][e] - st.base[0]),
                               abs(after["base_z"][e] - st.base[1])],
                 "yaw_rad": [ang_diff(after["yaw"][e], st.base[2])],
                 "joints_rad": np.abs(after["q"][:, e] - np.array(list(st.q))),
                 "tool_tip_m": np.abs(pose[e, 11:14] - np.array(list(o.ee)))}
        so = O.Oracle.state_objs(st)
        parts["objects_m"] = np.abs(after["obj"][e, :M, :4] - so).ravel()
        parts["obj_pos_out_m"] = np.abs(objo[e, :M] - so).ravel()
        if st.held >= 0:
            parts["attach_off_m"] = np.abs(after["c_off"][:, e] - np.array(list(st.c_off)))
            parts["pre_grasp_m"] = np.abs(after["p_pre"][:, e] - np.array(list(st.p_pre)))
            if boxes:
                parts["carried_rot"] = np.abs(after["r_off"][:, e] - np.array(list(st.r_off)))
        if boxes:
            sb = O.Oracle.state_boxes(st)
            gb = after["box"][e, :M]
            parts["box_extents_m"] = np.abs(gb[:, :3] - sb[:, :3]).ravel()
            parts["box_yaw_rad"] = [ang_diff(float(gb[j, 3]), float(sb[j, 3])) for j in range(M)]
        errs = []
        for k, v in parts.items():
            tally.note(k, v)
            errs += list(np.ravel(v))
        m = float(max(errs))
        tally.max_pose_err = max(tally.max_pose_err, m)
        assert m <= POSE_TOL, (e, m)
        assert pose[e, 7] == (1.0 if st.held >= 0 else 0.0)
        assert pose[e, 14] == st.step_count
        if reward is not None:
            # the task epilogue: reward, success and egomotion observations
            assert succ[e] == o.success, (e, succ[e], o.success)
            r_err = abs(float(reward[e]) - o.reward)
            obs_err = np.abs(tobs[e] - np.array(list(o.task_obs)))
            ts_err = np.abs(after["task"][e, :15] - np.array(
                [*st.goal, *st.obj_start, *st.prev_a, st.prev_d, st.prev_e]))
            tally.note("reward", r_err)
            tally.note("task_obs", obs_err)
            tally.note("task_state", ts_err)
            m2 = float(max([r_err, *obs_err, *ts_err]))
            tally.max_task_err = max(tally.max_task_err, m2)
            assert m2 <= POSE_TOL, (e, m2)


def oracle_image(orc, after, e, W, H, M, boxes=False):
    """The oracle's image of environment e's state: depth, RGB, ambiguity
    mask, |cos| of the winning hit, robot-body mask, counters."""
    st = oracle_state(after, e, M, boxes)
    cosv = np.ones((H, W))
    depth, rgb, amb, win, stats = orc.render(st, W, H, cos_out=cosv)
    robot = win >= orc.scene.n_tris + ROBOT_SLOT0 * (orc.objmesh.n_tris if orc.objmesh else 0)
    return depth, rgb, amb, cosv, robot, stats


def check_image(orc, after, out, e, W, H, M, tally, fp16=False, ref=None, boxes=False):
    """One image against the oracle's (ref: a precomputed oracle_image)."""
    depth, rgb, amb, cosv, robot, stats = ref if ref is not None else oracle_image(
        orc, after, e, W, H, M, boxes)
    gd = out["depth"][e].float().cpu().numpy().astype(np.float64)
    ok = ~amb
    tally.pixels += int(ok.sum())
    tally.ambiguous += int(amb.sum())
    cov_bad = int(((gd > 0) != (depth > 0))[ok].sum())
    tally.note("coverage_mismatch_px", cov_bad)
    assert cov_bad == 0, (e, cov_bad)
    if out.get("rgb") is not None:
        g = out["rgb"][e].cpu().numpy().astype(np.uint32)
        grgb = (g[..., 0] << 16) | (g[..., 1] << 8) | g[..., 2]
        bad = ok & (grgb != rgb)
        tally.note("rgb_mismatch_px", int(bad.sum()))
        assert not bad.any(), (e, int(bad.sum()))
    cov = ok & (depth > 0)
    if fp16:
        ulp = np.spacing(depth[cov].astype(np.float16)).astype(np.float64)
        lim = 0.5 * ulp + DEPTH_REL * depth[cov]
        err = np.abs(gd[cov] - depth[cov])
        tally.note("depth_fp16_m", err)
        if err.size:
            tally.fp16_max_err = max(tally.fp16_max_err, float(err.max()))
            tally.fp16_max_frac = max(tally.fp16_max_frac, float((err / lim).max()))
        assert np.all(err <= lim), (e, float((err - lim).max()))
    else:
        err = np.abs(gd[cov] - depth[cov])
        rel = err / depth[cov]
        tally.note("depth_fp32_m", err)
        tally.note("depth_fp32_rel", rel)
        if rel.size:
            tally.max_depth_rel = max(tally.max_depth_rel, float(rel.max()))
        rob = robot[cov]
        tally.robot_pixels += int(rob.sum())
        lim = DEPTH_REL * depth[cov] + np.where(rob, DEPTH_ABS / np.maximum(cosv[cov], 0.05), 0.0)
        if (~rob).any():
            tally.note("depth_fp32_rel_scene", rel[~rob])
        assert np.all(err <= lim), (e, float((err - lim).max()))
    return stats
