#!/usr/bin/env python
"""DPA-1 E+F(+virial) throughput on one GB300 per rank.

Workload: the 15,668-atom solvated-protein-like periodic box (jittered
lattice at 0.1 atoms/A^3, elemental fractions H .63 C .12 N .03 O .21
S .01, seed 1) with the default DPA-1 model (5 types, type embedding 8,
rcut 6 A, sel 120, embedding [25,50,100], axis 16, 2 gated attention
layers of width 128, fitting [240,240,240], seed-0 Xavier weights).

A step is one evaluation of the whole path: cell list and neighbour list,
environment matrix, embedding, attention, descriptor, fitting, FP64 energy
sum, the hand-written adjoint and the force / virial reduction.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun every rank evaluates its own replica of the box (weak
scaling, no collective on the data path); the timing is the maximum over
ranks.  ``--impl reference`` times the FP64 CPU oracle on bounded samples
of the same workload instead.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DPA-1 E+F atom-steps/s at 15,668 atoms, BF16 vs FP32, force RMSE vs FP64"
NATOMS = 15668
def workload(natoms):
    return f"solvated-protein-like periodic box, {natoms:,} atoms, jittered lattice at 0.1/A^3, seed 1"
MODEL = ("DPA-1 se_atten: 5 types, tebd 8, rcut 6.0/0.5 A, sel 120, embed [25,50,100], axis 16, "
         "2 gated attention layers x 128, fitting [240,240,240]")
# --model: the measured model (default) and the widened variants; weights are
# seeded, as for the default
MODELS = {
    "dpa1": (MODEL, {}),
    "paper-size": ("DPA-1 se_atten at the paper's size: 5 types, tebd 8, rcut 6.0/0.5 A, sel 120, embed [32,64,128], "
                   "axis 16, 3 gated attention layers x 256, fitting [256,256,256] (bf16x and FP32 paths)",
                   dict(embed=(32, 64, 128), attn_layers=3, attn_dim=256, fitting=(256, 256, 256))),
    "concat": ("DPA-1 se_atten, concat type embedding (embedding net input [s, T_j, T_i]); otherwise the default "
               "model", dict(tebd_input_mode="concat")),
}


def model_cfg(name):
    import dataclasses

    import synth

    desc, kw = MODELS[name]
    # the paper-size model has its own calibrated output scale
    base = synth.PAPER_SIZE_CONFIG if name == "paper-size" else synth.DEFAULT_CONFIG
    return dataclasses.replace(base, **kw), desc


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp16x", "bf16x", "bf16", "fp32"])
    ap.add_argument("--natoms", type=int, default=NATOMS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=12288,
                    help="oracle centres timed for cpu_baseline (about 11 s on 16 cores)")
    ap.add_argument("--ref-sample", type=int, default=512, help="oracle centres per --impl reference step")
    ap.add_argument("--md-steps", type=int, default=1000, help="graph-captured velocity-Verlet steps to time (0: skip)")
    ap.add_argument("--no-student", action="store_true", help="skip the distilled-student line")
    ap.add_argument("--student-frames", type=int, default=0,
                    help="also run the student configuration at full size with this many teacher frames of the "
                         "measured box (20000: about 15 minutes; 0: skip)")
    ap.add_argument("--model", default="dpa1", choices=sorted(MODELS), help="dpa1: the measured model")
    ap.add_argument("--no-batch", action="store_true", help="skip the 32-frame dp_compute_batch line")
    ap.add_argument("--scale-natoms", type=int, default=250000,
                    help="atoms of the scale box timed after the main line (fp16x; 0: skip)")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, device):
    """Largest value of x over the ranks of the default process group (x
    itself without one): the job's time is its slowest replica's."""
    import torch
    import torch.distributed as td

    if not (td.is_available() and td.is_initialized()) or td.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, natoms, steps, seconds):
    """Whole-job throughput: every replica's atom-steps over the slowest
    replica's time (weak scaling, one box per GPU)."""
    return world * natoms * steps / seconds


def _system(natoms):
    import synth

    coord, atype, box = synth.lattice_system(natoms, seed=1)
    return coord, atype, box


# ----------------------------------------------------------------- oracle arm

def _oracle_sample_rate(coord, atype, box, sample, seed=0, model="dpa1"):
    """Atom-steps/s of the FP64 oracle: energy and forces of ``sample``
    centres (their atomic energies and the gradient they contribute)."""
    import torch

    import synth
    from oracle import OracleModel, energy_force_virial

    cfg, _ = model_cfg(model)
    om = OracleModel.from_numpy(cfg, synth.make_weights(cfg, seed=0))
    rng = np.random.default_rng(seed)
    centres = np.sort(rng.choice(len(coord), size=min(sample, len(coord)), replace=False))
    t0 = time.perf_counter()
    energy_force_virial(om, coord, box, atype, centres=centres)
    dt = time.perf_counter() - t0
    return len(centres) / dt, dt, torch.get_num_threads()


def run_reference(a):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    coord, atype, box = _system(a.natoms)
    vals = []
    for s in range(a.warmup + a.steps):
        v, dt, cores = _oracle_sample_rate(coord, atype, box, a.ref_sample, seed=s, model=a.model)
        if s >= a.warmup:
            vals.append((v, dt))
    rate = len(vals) * a.ref_sample / sum(dt for _, dt in vals)
    sample = f"{a.ref_sample} random centres of the {a.natoms}-atom box per step (E, e_i and their force terms)"
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "atom-steps/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * sum(dt for _, dt in vals) / len(vals),
        "ms_per_step_is": f"the oracle's time for one {a.ref_sample}-centre sample, not for a whole {a.natoms}-atom step "
                          f"(about {a.natoms / rate:.0f} s at this rate)",
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload(a.natoms), "model": model_cfg(a.model)[1], "natoms": a.natoms},
        "cpu_baseline": {"value": rate, "unit": "atom-steps/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": "atom-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------------- our arm

def _student_line(dev, coord, atype, box, full_rates, batch=16, md_steps=100):
    """The distilled student (embedding [16, 32, 64], axis 8, no attention,
    fitting [128, 128]) and its teacher (the same sizes with one gated
    attention layer of small LayerNorm gain, synth.teacher_weights).

    On the measured box: teacher frame generation (velocity-Verlet at 10 K,
    a frame every 2 steps), training throughput of dp_train_frame +
    dp_adam_step on 16-frame batches with FP32 products and with the fitting
    net as BF16 two-term splits on the tensor cores (bf16x), and MD
    throughput of student, teacher and the full default model.  On the
    water box (where 10 K trajectories stay physical for a random-weight
    potential): training from perturbed weights to the family's floor and
    MD with the full-model check at 0.05 eV/A."""
    import torch

    import synth
    import paper_2604_07276_gb300 as dp
    from paper_2604_07276_gb300 import md as dmd, student as stu

    d = tempfile.mkdtemp(prefix="dpa1s_")
    tcfg, tw = synth.teacher_weights(ln_gain=3e-3)
    scfg, bw = synth.teacher_base_weights(synth.TEACHER_BASE_OUT_SCALE)
    sw = synth.perturbed(bw, 0.03, seed=21)
    tpath, bpath, spath = (os.path.join(d, f) for f in ("teacher.bin", "base.bin", "student.bin"))
    synth.write_weights(tpath, tcfg, tw)
    synth.write_weights(bpath, scfg, bw)
    synth.write_weights(spath, scfg, sw)
    n = len(coord)
    out = {"student": "embed [16,32,64], axis 8, no attention, fitting [128,128]",
           "teacher": "the student's sizes plus one gated attention layer (width 128, LayerNorm gain 3e-3)",
           "box_atoms": n}

    # teacher frames on the measured box (10 K, dt 0.25 fs, a frame every 2 steps)
    teacher = dp.DPA1(tpath, precision="fp16x", device=dev.index)
    t0 = time.perf_counter()
    frames = stu.teacher_frames(teacher, [(coord, atype, box)], synth.MASSES, n_traj=2, steps=2 * batch, every=2,
                                dt=0.25, temperature=10.0, seed=1)
    torch.cuda.synchronize(dev)
    gen_s = time.perf_counter() - t0
    out["teacher_frames_per_s"] = len(frames) / gen_s
    train_rate = {}
    for prec in ("fp32", "bf16x"):
        s = dp.DPA1(spath, precision=prec, device=dev.index)
        stu.train(s, frames[:batch], epochs=1, batch=batch, lr0=1e-6, lr_end=1e-6)  # warm-up
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        stu.train(s, frames, epochs=1, batch=batch, lr0=1e-6, lr_end=1e-6)
        torch.cuda.synchronize(dev)
        train_rate[prec] = len(frames) / (time.perf_counter() - t0)
        s.close()
    out["train_batch_frames"] = batch
    out["train_frames_per_s"] = train_rate
    # the configuration's 20,000-frame run, extrapolated from the measured rates
    out["hours_for_20000_frames_extrapolated"] = {
        "generate": 20000 / out["teacher_frames_per_s"] / 3600,
        "train_one_epoch_bf16x": 20000 / train_rate["bf16x"] / 3600}

    def md_rate(path, precision):
        mdl = dp.DPA1(path, precision=precision, device=dev.index)
        mdl.reserve(n)
        state = dmd.MDState(coord, np.zeros_like(coord), synth.MASSES[atype], box, atype, device=dev)
        dmd.run(mdl, state, dt=0.25, nsteps=2, graph=True)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        dmd.run(mdl, state, dt=0.25, nsteps=md_steps, graph=True)
        e1.record()
        torch.cuda.synchronize(dev)
        mdl.status()
        mdl.close()
        return n * md_steps / (e0.elapsed_time(e1) / 1e3)

    teacher.close()
    rates = {"student_fp16x": md_rate(spath, "fp16x"), "student_fp32": md_rate(spath, "fp32"),
             "teacher_fp16x": md_rate(tpath, "fp16x")}
    out["md_atom_steps_per_s"] = rates
    if "fp16x" in full_rates:
        out["md_speedup_vs_full_fp16x"] = rates["student_fp16x"] / full_rates["fp16x"]
    out["md_speedup_vs_teacher_fp16x"] = rates["student_fp16x"] / rates["teacher_fp16x"]

    # accuracy at the threshold: the water-box distillation
    teacher = dp.DPA1(tpath, precision="fp32", device=dev.index)
    base = dp.DPA1(bpath, precision="fp32", device=dev.index)
    systems = [synth.water_box(k) for k in range(3)]
    wf = stu.teacher_frames(teacher, systems, synth.MASSES, n_traj=6, steps=8, every=2, dt=0.25, temperature=10.0,
                            seed=1)
    held = stu.teacher_frames(teacher, systems, synth.MASSES, n_traj=2, steps=8, every=4, dt=0.25, temperature=10.0,
                              seed=2)
    acc = {"floor_force_rmse": stu.force_rmse(base, held)}
    for prec in ("fp32", "bf16x"):
        s = dp.DPA1(spath, precision=prec, device=dev.index)
        s0 = dp.DPA1(spath, precision=prec, device=dev.index)
        before = stu.force_rmse(s, held)
        stu.train(s, wf, epochs=60, batch=8, lr0=1e-5, lr_end=1e-6)
        c, t, b = synth.water_box(1)
        vel = synth.maxwell_boltzmann(t, 10.0, seed=33)
        runs = {}
        for name, mdl in (("trained", s), ("untrained", s0)):
            st = dmd.MDState(c, vel, synth.MASSES[t], b, t)
            u_s, u_t, _ = stu.md_with_fallback(mdl, teacher, st, nsteps=12, dt=0.25, check_every=3, threshold=0.05)
            runs[name] = {"student_segments": u_s, "fallback_segments": u_t}
        acc[prec] = {"held_out_force_rmse_before": before, "held_out_force_rmse_after": stu.force_rmse(s, held),
                     "md_at_0.05": runs}
        s.close()
        s0.close()
    teacher.close()
    base.close()
    acc["frames"] = {"train": len(wf), "held_out": len(held), "system": "three 192-atom water boxes, 10 K"}
    out["distillation"] = acc
    return out


def _student_config_line(dev, coord, atype, box, nframes, batch=16, held_traj=25):
    """The distilled-student configuration at full size: ``nframes`` teacher
    frames of the measured box from full-model MD (fp16x; 2 fs trajectories at
    10 K from fresh Maxwell-Boltzmann draws, dt 0.25 fs, a frame every 2
    steps), all held in device memory; one epoch of training in batches of
    ``batch`` frames with the fitting net's products as BF16 two-term splits
    (bf16x); the held-out force error before and after against the family's
    floor; and student MD on the box with the full-model check every 10 steps
    at 0.05 eV/A, trained against untrained."""
    import math

    import torch

    import synth
    import paper_2604_07276_gb300 as dp
    from paper_2604_07276_gb300 import md as dmd, student as stu

    d = tempfile.mkdtemp(prefix="dpa1sc_")
    tcfg, tw = synth.teacher_weights(ln_gain=3e-3)
    scfg, bw = synth.teacher_base_weights(synth.TEACHER_BASE_OUT_SCALE)
    sw = synth.perturbed(bw, 0.03, seed=21)
    tpath, bpath, spath = (os.path.join(d, f) for f in ("teacher.bin", "base.bin", "student.bin"))
    synth.write_weights(tpath, tcfg, tw)
    synth.write_weights(bpath, scfg, bw)
    synth.write_weights(spath, scfg, sw)
    n = len(coord)
    teacher = dp.DPA1(tpath, precision="fp16x", device=dev.index)
    free0 = torch.cuda.mem_get_info(dev)[0]
    t0 = time.perf_counter()
    frames = stu.teacher_frames(teacher, [(coord, atype, box)], synth.MASSES, n_traj=math.ceil(nframes / 4), steps=8,
                                every=2, dt=0.25, temperature=10.0, seed=1)[:nframes]
    torch.cuda.synchronize(dev)
    gen_s = time.perf_counter() - t0
    frames_bytes = free0 - torch.cuda.mem_get_info(dev)[0]
    held = stu.teacher_frames(teacher, [(coord, atype, box)], synth.MASSES, n_traj=held_traj, steps=8, every=4,
                              dt=0.25, temperature=10.0, seed=2)
    out = {"frames": len(frames), "box_atoms": n, "batch": batch, "held_out_frames": len(held),
           "generate_s": gen_s, "generate_frames_per_s": len(frames) / gen_s,
           "frames_device_bytes": frames_bytes}
    base = dp.DPA1(bpath, precision="fp32", device=dev.index)
    out["floor_force_rmse"] = stu.force_rmse(base, held)
    base.close()
    s = dp.DPA1(spath, precision="bf16x", device=dev.index)
    s0 = dp.DPA1(spath, precision="bf16x", device=dev.index)
    out["held_out_force_rmse_before"] = stu.force_rmse(s, held)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    hist = stu.train(s, frames, epochs=1, batch=batch, lr0=1e-5, lr_end=1e-6)
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    out["train_s"] = train_s
    out["train_frames_per_s"] = len(frames) / train_s
    out["adam_steps"] = len(hist)
    out["loss_first_last_batch"] = [float(hist[0][0]), float(hist[-1][0])]
    out["held_out_force_rmse_after"] = stu.force_rmse(s, held)
    del frames
    vel = synth.maxwell_boltzmann(atype, 10.0, seed=33)
    runs = {}
    for name, mdl in (("trained", s), ("untrained", s0)):
        st = dmd.MDState(coord, vel, synth.MASSES[atype], box, atype)
        u_s, u_t, checks = stu.md_with_fallback(mdl, teacher, st, nsteps=40, dt=0.25, check_every=10,
                                                threshold=0.05)
        runs[name] = {"student_segments": u_s, "fallback_segments": u_t, "check_force_rmse": checks}
    out["md_at_0.05"] = {"steps": 40, "dt_fs": 0.25, "check_every": 10, **runs}
    s.close()
    s0.close()
    teacher.close()
    return out


def _scale_line(a, dev, cfg, wpath, steps=5):
    """The scale configuration: the same recipe at a.scale_natoms atoms (seed
    4), fp16x, device-resident inputs; step time, device memory of the model
    and sampled parity against the oracle (exact forces on 4 atoms from the
    atomic energies of the centres that depend on them)."""
    import torch

    import synth
    import paper_2604_07276_gb300 as dp

    n = a.scale_natoms
    coord, atype, box = synth.lattice_system(n, seed=4)
    torch.cuda.synchronize(dev)
    free0 = torch.cuda.mem_get_info(dev)[0]
    m = dp.DPA1(wpath, precision="fp16x", device=dev.index)
    m.reserve(n)
    torch.cuda.synchronize(dev)
    mem = free0 - torch.cuda.mem_get_info(dev)[0]
    c = torch.tensor(coord, dtype=torch.float64, device=dev)
    t = torch.tensor(atype, dtype=torch.int32, device=dev)
    b = torch.tensor(dp.box9(box), dtype=torch.float64, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    F = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    W = torch.zeros(9, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    for _ in range(2):
        m.compute_device(c, b, t, E, F, W, stream=stream.cuda_stream)
    torch.cuda.synchronize(dev)
    m.status()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        m.compute_device(c, b, t, E, F, W, stream=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    m.status()
    ms = e0.elapsed_time(e1) / steps
    line = {"natoms": n, "precision": "fp16x", "steps": steps, "ms_per_step": ms, "atom_steps_per_s": n / (ms / 1e3),
            "device_memory_bytes": mem, "workload": workload(n).replace("seed 1", "seed 4")}
    if not a.no_parity:
        from oracle import OracleModel, energy_force_virial, reverse_centres

        _, Fh, _, eh = m.compute(coord, box, atype, atom_energy=True)
        om = OracleModel.from_numpy(cfg, synth.make_weights(cfg, seed=0))
        atoms = np.sort(np.random.default_rng(9).choice(n, size=4, replace=False))
        cs = reverse_centres(coord, box, cfg.rcut, cfg.sel, atoms)
        _, e_ref, f_ref, _ = energy_force_virial(om, coord, box, atype, centres=cs)
        line["sampled_parity"] = {"force_rmse_ev_per_A": float(np.sqrt(np.mean((Fh[atoms] - f_ref[atoms]) ** 2))),
                                  "atoms": len(atoms),
                                  "atomic_energy_max_abs_err_eV": float(np.abs(eh[cs] - e_ref).max()),
                                  "centres": int(len(cs)),
                                  "sum_of_forces_max_abs": float(np.abs(Fh.sum(axis=0)).max())}
    m.close()
    return line


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons (every 100 ms).
    ``mark()`` is called as the timed region starts; only samples written
    after it count."""

    def __init__(self, index):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        self.start_line = 0
        # the sampler is running once its first line is out (bounded wait)
        t0 = time.time()
        while self.p is not None and self._lines() == 0 and time.time() - t0 < 5.0 and self.p.poll() is None:
            time.sleep(0.02)

    def _lines(self):
        try:
            with open(self.path) as fh:
                return sum(1 for _ in fh)
        except OSError:
            return 0

    def mark(self):
        self.start_line = self._lines()

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        self.p.wait()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = open(self.path).read().splitlines()
        if len(lines) > self.start_line:
            lines = lines[self.start_line:]
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# ncu summary that holds the DRAM traffic of a stage's kernel, per atom
TRAFFIC_PROFILES = {"attn_bwd_tc": ("profiles/k_layer_bwd_tc_fp16x_2000atoms.md", "paper_2604_07276_gb300/csrc/tc.cu")}


def _traffic_per_launch(stage, natoms):
    """dram__bytes_read.sum + dram__bytes_write.sum of one launch, scaled from
    the committed ncu capture by the atoms processed; None when there is no
    capture or the kernel source changed since it was taken."""
    import hashlib

    if stage not in TRAFFIC_PROFILES:
        return None
    prof, src = (os.path.join(ROOT, x) for x in TRAFFIC_PROFILES[stage])
    try:
        text = open(prof).read()
        want = text.split("source sha256 (csrc/tc.cu):")[1].split()[0]
        per_atom = float(text.split("dram bytes per atom:")[1].split()[0])
        have = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except (OSError, IndexError, ValueError):
        return None
    return per_atom * natoms if have.startswith(want) else None


def _flops_per_launch(stage, nn, cfg):
    """Algorithmic FLOPs of one launch of ``stage`` over the whole box
    (per attention layer for per-layer stages), from the real neighbour
    counts n_i: attention core forward 2 n^2 A MAC, backward 4 n^2 A MAC,
    projections per neighbour row 3 A M1 (QKV) and A M1 (output)."""
    A, m1 = cfg.attn_dim, cfg.m1
    n2 = float(np.sum(nn.astype(np.float64) ** 2))
    n1 = float(np.sum(nn))
    proj = 4 * A * m1  # Q, K, V and output projections per neighbour row
    table = {
        "attn_fwd": 2 * n2 * A,
        "attn_bwd": 4 * n2 * A,
        "attn_fwd_tc": proj * n1 + 2 * n2 * A,  # a whole fused layer
        "attn_bwd_tc": proj * n1 + 4 * n2 * A,
        "qkv_gemm": n1 * 3 * A * m1,
        "qkv_bwd_gemm": n1 * 3 * A * m1,
    }
    mac = table.get(stage)
    return None if mac is None else 2.0 * mac


def run_ours(a):
    import torch

    import synth
    import paper_2604_07276_gb300 as dp

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as tdist

        tdist.init_process_group(backend="nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg, model_desc = model_cfg(a.model)
    wpath = os.path.join(tempfile.mkdtemp(prefix=f"dpa1b{rank}_"), "w.bin")
    synth.write_weights(wpath, cfg, synth.make_weights(cfg, seed=0))
    coord, atype, box = _system(a.natoms)
    n = len(coord)

    precisions = ["fp16x", "bf16x", "bf16", "fp32"] if a.precision == "auto" else [a.precision]
    models = {}
    mem_used = {}  # device bytes taken by each model (weights + workspace for n atoms)
    for p in precisions:
        try:
            torch.cuda.synchronize(dev)
            free0 = torch.cuda.mem_get_info(dev)[0]
            models[p] = dp.DPA1(wpath, precision=p, device=local)
            models[p].reserve(n)
            torch.cuda.synchronize(dev)
            mem_used[p] = free0 - torch.cuda.mem_get_info(dev)[0]
        except dp.DPError as e:
            if e.code != -8 or a.precision != "auto":
                raise
    head = next(p for p in ("fp16x", "bf16x", "bf16", "fp32") if p in models)

    c = torch.tensor(coord, dtype=torch.float64, device=dev)
    t = torch.tensor(atype, dtype=torch.int32, device=dev)
    b = torch.tensor(dp.box9(box), dtype=torch.float64, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    F = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    W = torch.zeros(9, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    results = {}
    for p, m in models.items():
        for _ in range(a.warmup):
            m.compute_device(c, b, t, E, F, W, stream=stream.cuda_stream)
        torch.cuda.synchronize(dev)
        m.status()
        clk = Clocks(local) if p == head else None
        barrier()
        torch.cuda.synchronize(dev)
        m.set_profiling(True)
        l0 = dp.kernel_launches()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        if clk:
            clk.mark()
        ev0.record(stream)
        for _ in range(a.steps):
            m.compute_device(c, b, t, E, F, W, stream=stream.cuda_stream)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        launches = dp.kernel_launches() - l0
        barrier()
        ms = ev0.elapsed_time(ev1)
        clocks = clk.stop() if clk else None
        stages = m.stage_times()
        m.set_profiling(False)
        m.status()
        ms = max_over_ranks(ms, dev)
        per_stage = {}
        for name, v in stages:
            s = per_stage.setdefault(name, [0.0, 0])
            s[0] += v
            s[1] += 1
        results[p] = {"ms": ms, "launches": launches, "clocks": clocks, "stages": per_stage}

    # e2e through the host-buffer entry point (pinned host memory)
    m = models[head]
    hc = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    hc[:] = coord
    ht = torch.empty(n, dtype=torch.int32, pin_memory=True).numpy()
    ht[:] = atype
    for _ in range(max(1, a.warmup // 2)):
        m.compute(hc, box, ht)
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(3, a.steps // 2)
    for _ in range(e2e_steps):
        m.compute(hc, box, ht)
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dev)

    # velocity-Verlet MD of the same box, every step replayed from one CUDA graph
    md_line = None
    if a.md_steps > 0:
        from paper_2604_07276_gb300 import md as dmd

        vel = synth.maxwell_boltzmann(atype, 300.0, seed=11)
        state = dmd.MDState(coord, vel, synth.MASSES[atype], box, atype, device=dev)
        dmd.run(m, state, dt=0.5, nsteps=2, graph=True, stream=stream.cuda_stream)  # capture + warm-up
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        th = dmd.run(m, state, dt=0.5, nsteps=a.md_steps, graph=True, stream=stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        md_status = "ok"
        try:
            m.status()
        except dp.DPError as e:  # e.g. a non-finite coordinate once atoms collapse
            md_status = str(e)
        md_ms = max_over_ranks(e0.elapsed_time(e1), dev)
        thc = th.cpu().numpy()
        md_line = {"steps": a.md_steps, "dt_fs": 0.5, "graph": True, "precision": head,
                   "atom_steps_per_s": job_rate(ws, n, a.md_steps, md_ms / 1e3), "ms_per_step": md_ms / a.md_steps,
                   "total_energy_drift_eV_per_atom_first_20_steps": float(abs(thc[min(19, len(thc) - 1), 2] - thc[0, 2]) / n),
                   "total_energy_drift_eV_per_atom_all_steps": float(abs(thc[-1, 2] - thc[0, 2]) / n),
                   "status": md_status,
                   "note": "random weights have no short-range repulsion; long runs collapse atoms"}

    batch = None
    if rank == 0 and not a.no_batch:
        # 32 independent frames of U{200..3000} atoms through dp_compute_batch
        # (host arrays, copies included), as a user of the batch call sees it
        frames = synth.frame_batch(seed=2, nframes=32)
        mb = models[head]
        mb.compute_batch(frames)
        reps = 5
        t0 = time.perf_counter()
        for _ in range(reps):
            mb.compute_batch(frames)
        dtb = (time.perf_counter() - t0) / reps
        natb = sum(len(t) for _, t, _ in frames)
        batch = {"frames": len(frames), "atoms": natb, "precision": head, "ms_per_batch": 1e3 * dtb,
                 "frames_per_s": len(frames) / dtb, "atom_steps_per_s": natb / dtb,
                 "api": "dp_compute_batch, host arrays (copies included)"}
    student = None
    if not a.no_student:
        student = _student_line(dev, coord, atype, box,
                                {p: job_rate(1, n, a.steps, rr["ms"] / 1e3) for p, rr in results.items()})
    if a.student_frames > 0:
        student = dict(student or {})
        student["configuration_run"] = _student_config_line(dev, coord, atype, box, a.student_frames)

    # parity of this run against the FP64 oracle over the whole box: every
    # atomic energy, every force, the total energy and the virial
    parity = {}
    nl, nn = m.nlist_device(c, b)
    nn = nn.cpu().numpy()
    if rank == 0 and not a.no_parity:
        from oracle import OracleModel, energy_force_virial

        om = OracleModel.from_numpy(cfg, synth.make_weights(cfg, seed=0))
        t0 = time.perf_counter()
        rE, e_ref, f_ref, w_ref = energy_force_virial(om, coord, box, atype)
        t_oracle = time.perf_counter() - t0
        for p, mm in models.items():
            Ep, Fp, Wp, ep = mm.compute(coord, box, atype, atom_energy=True)
            parity[p] = {"force_rmse_ev_per_A": float(np.sqrt(np.mean((Fp - f_ref) ** 2))),
                         "force_max_abs_err_ev_per_A": float(np.abs(Fp - f_ref).max()),
                         "atomic_energy_max_abs_err_eV": float(np.abs(ep - e_ref).max()),
                         "atomic_energy_rms_err_eV": float(np.sqrt(np.mean((ep - e_ref) ** 2))),
                         "energy_abs_err_eV_per_atom": abs(Ep - rE) / n,
                         "virial_max_rel_err": float(np.abs(Wp - w_ref).max() / np.abs(w_ref).max()),
                         "atoms_compared": n,
                         "within_16bit_bounds": bool(np.sqrt(np.mean((Fp - f_ref) ** 2)) <= 5e-3
                                                     and np.abs(ep - e_ref).max() <= 1e-3),
                         "within_fp32_bound": bool(np.sqrt(np.mean((Fp - f_ref) ** 2)) <= 1e-5)}
        parity["oracle_seconds"] = t_oracle

    scale = None
    if rank == 0 and a.scale_natoms > 0 and "fp16x" in models:
        for mm in models.values():
            mm.close()
        models.clear()
        scale = _scale_line(a, dev, cfg, wpath)

    if rank != 0:
        return 0
    r = results[head]
    ms_step = r["ms"] / a.steps
    value = job_rate(ws, n, a.steps, r["ms"] / 1e3)
    # dominant kernel stage and its roofline
    peaks = _peaks()
    st = r["stages"]
    dom = max(st.items(), key=lambda kv: kv[1][0])[0]
    dom_avg_ms = st[dom][0] / st[dom][1]
    flops = _flops_per_launch(dom, nn, cfg)
    roof = None
    if flops is not None:
        achieved = flops / (dom_avg_ms / 1e3) / 1e12
        if head in ("bf16", "fp16x", "bf16x"):
            # FP16 and BF16 share the nominal dense rate: the measured BF16 figure applies
            # a kernel of a few ms inside a sub-second timed region: the burst peak
            peak = (peaks or {}).get("bf16_tflops", 1900.0)
            roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": _traffic_per_launch(dom, n), "kernel": dom,
                    "peak_source": "measured bf16 burst" if peaks else "fallback"}
        else:
            clock = (peaks or {}).get("sm_max_mhz", 2070.0)
            peak = 152 * 128 * 2 * clock * 1e6 / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": None, "kernel": dom,
                    "peak_source": "152 SMs x 128 FP32 lanes x 2 FLOP x max SM clock"}
    cpu = None
    if not a.no_cpu_baseline and ws == 1:
        v, dt, cores = _oracle_sample_rate(coord, atype, box, a.cpu_sample, model=a.model)
        cpu = {"value": v, "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
               "sample": f"{a.cpu_sample} random centres of the {n}-atom box (E, e_i and their force terms), {dt:.1f} s"}
    h2d = n * 3 * 8 + n * 4 + 9 * 8
    d2h = 8 + 9 * 8 + n * 3 * 8
    line = {
        "metric": METRIC, "value": value, "unit": "atom-steps/s", "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp16x": "f16", "bf16x": "bf16", "bf16": "bf16", "fp32": "f32"}[head],
        "data": "synthetic",
        "config": {"workload": workload(n), "model": model_desc, "natoms": n, "global_batch": ws * n,
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": "per-step working set is several GB of intermediates, far above the 129 MB L2",
                   "arithmetic": {"fp16x": "attention layers, embedding and fitting nets on tcgen05: FP16 operands, "
                                           "two-term splits of G, P and the weights (Y = P [G 1] [Wv Wo; bv Wo]); "
                                           "FP32 accumulation; FP64 energy / virial sums",
                                  "bf16x": "attention layers, embedding and fitting nets on tcgen05: BF16 operands with "
                                           "two-term splits of both operands, FP32 accumulation; FP64 energy / "
                                           "virial sums",
                                  "bf16": "attention layers on tcgen05: plain BF16 operands, FP32 accumulation",
                                  "fp32": "FP32 SIMT"}[head]},
        "clocks": r["clocks"],
        "e2e": {"value": job_rate(ws, n, e2e_steps, e2e_s), "unit": "atom-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": r["launches"],
        "roofline": roof,
        "cpu_baseline": cpu,
        "precisions": {p: {"value": job_rate(ws, n, a.steps, rr["ms"] / 1e3), "ms_per_step": rr["ms"] / a.steps}
                       for p, rr in results.items()},
        "force_rmse_vs_fp64": parity,
        "bf16_vs_fp32": ({"bf16_operand_mode": "bf16x",
                          "ms_per_step": {"bf16x": results["bf16x"]["ms"] / a.steps, "fp32": results["fp32"]["ms"] / a.steps},
                          "speedup": results["fp32"]["ms"] / results["bf16x"]["ms"],
                          "within_16bit_bounds": parity.get("bf16x", {}).get("within_16bit_bounds")}
                         if "bf16x" in results and "fp32" in results else None),
        "stage_ms_per_step": {p: {k: v[0] / a.steps for k, v in rr["stages"].items()} for p, rr in results.items()},
        "neighbors": {"mean": float(nn.mean()), "max": int(nn.max())},
        "device_memory_bytes": mem_used,
        "md": md_line,
        "student": student,
        "batch": batch,
        "scale": scale,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    a = _args()
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
