#!/usr/bin/env python3
"""Benchmark: the 28-qubit diagonal-heavy gate-level stream on one GB300.

One step = simulate the whole circuit from |0...0>: reset + optimizer
(diagonal detector, gate-block search, fusion) + every kernel of the plan,
over a 2 GiB complex64 state resident in HBM (larger than the 129 MB L2, so
no flush is needed between steps).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (torchrun): independent replicas, one per GPU (the path does not
shard: replicas only); value = total amplitude updates of all ranks / the
slowest rank's time.  ``--impl reference`` times the CPU oracle (the only
reference this paper has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "amplitude-updates/s & HBM GB/s vs peak; served circuits/s, p50/p99 latency"
UNIT = "amplitude-updates/s"
N_QUBITS = 28
N_GATES = 500
SEED = 1
WORKLOAD = "28-qubit diagonal-heavy gate-level stream (500 gates, 80% RZ/CP/RZZ, 20% H/RX, after H on every qubit), complex64"

# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of
# the dominant kernel, per amplitude, keyed by (workload, op kind, sha256 of
# the kernel's source file at capture time): null once the kernel changed.
# A sweep's traffic grows with the amplitudes it processes, so a capture on a
# smaller state scales to the full one (profiles/ has the captures).
TRAFFIC_PER_AMP = {
    # profiles/svs_chunk_jit_diagheavy_28q.md: 3.9241 GB per launch, the mean of
    # one step's seven 2^28-amplitude sweeps (six read + write, one write-only)
    # at this workload's own size, as `achieved` averages the algorithmic bytes
    # (the specialised kernel: keyed by its device templates and generator)
    ("diag-heavy", "chunk-jit", "b550109b50cf382e660da46a21662018df0103984dbd8174814aed752c456a33"): 3.92412e9 / 2 ** 28,
    # profiles/k_chunk_diagheavy_25q.md: 476.05 MB per 2^25-amplitude sweep (interpreter)
    ("diag-heavy", "chunk", "8f96366b3d7184491700fbf33588aba4d28412cc874eee7e00ed69b7789963a2"): 476.05e6 / 2 ** 25,
    # profiles/k_dense5_tc_layered_26q.md: 1011.84 MB per 2^26-amplitude block sweep
    ("layered-dense", "dense", "902dcf26ad8abd672acf4f9ec16df78b31986b3b9a62774a4456ee0248f2943f"): 1011.84e6 / 2 ** 26,
    # profiles/svs_diag_jit_rzzfull_26q.md: 475.18 MB per write-only 2^26-amplitude sweep
    ("rzz-full", "diag-jit", "359062f70d7e6966f803d6dcbb4c08f0795e984a9309e29795f9a2ea43905579"): 475.18e6 / 2 ** 26,
    # profiles/k_diag_rzzfull_26q.md: 475.29 MB per write-only 2^26-amplitude sweep (interpreter)
    ("rzz-full", "diag", "8f96366b3d7184491700fbf33588aba4d28412cc874eee7e00ed69b7789963a2"): 475.29e6 / 2 ** 26,
}


def max_over_ranks(x: float, dist=None) -> float:
    """The largest x over all ranks (the slowest rank's time); x itself
    without a process group.  NCCL reduces a device tensor, gloo a host one."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput of N independent replicas (weak scaling): the
    units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / seconds_max


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for i, nm in enumerate(names):
                if f[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


PRECISIONS = {"tf32x3": 0, "fp32": 1, "fp64": 2, "df": 3}
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12     # SMs x FP32 lanes x FMA x max SM clock
TF32_PER_BF16 = 1.1 / 2.25                             # nominal dense TF32 / BF16 tensor rates of a GB300
TF32_FLOPS_PER_AMP_BLOCK = 3 * 2 * 64 * 64 / 32        # split-TF32: three 64 x 64 real products per 32 amplitudes


def _tf32_peak(sustained=True):
    """Dense TF32 tensor peak: the measured cuBLAS bf16 figure (sustained for
    a kernel timed inside a long step) times the nominal TF32/BF16 ratio."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        key = "bf16_tflops_sustained" if sustained and "bf16_tflops_sustained" in d else "bf16_tflops"
        if key in d:
            return d[key] * TF32_PER_BF16, f"measured {key} x {TF32_PER_BF16:.3f} (nominal TF32/BF16)"
    return (1700.0 if sustained else 1900.0) * TF32_PER_BF16, "fallback bf16 x nominal TF32/BF16"
DF_FLOPS_PER_AMP = 2 * 64 * 15 + 2 * 3                 # double-float complex128 dense block
DF_OPS_PER_FLOP = 7.5                                  # FP32 operations per double-float flop (15 per multiply-add)


def _redraw(c, seed):
    """The circuit with the same gates on the same qubits and every angle
    (uniform in [0, 2 pi)) and Haar one-qubit matrix drawn anew."""
    import numpy as np
    from paper_2604_12256_gb300 import circuits as C
    rng = np.random.default_rng(seed)
    gs = []
    for g in c.gates:
        if g.kind == "u1q":
            gs.append(C.Gate("u1q", g.qubits, matrix=C.haar_u2(rng)))
        elif g.params:
            gs.append(C.Gate(g.kind, g.qubits, tuple(float(rng.uniform(0, 2 * math.pi)) for _ in g.params)))
        else:
            gs.append(g)
    return C.Circuit(c.n, gs, c.basis, c.name)


def _workload_circuit(args, n):
    from paper_2604_12256_gb300 import circuits as C
    if args.workload in ("layered-dense", "layered"):
        return C.layered(n, 20, 0)
    if args.workload == "rzz-full":
        return C.rzz_full(n)
    if args.workload == "qft":
        return C.qft(n, 2)
    if args.workload == "qaoa":
        return C.qaoa(n, 4, 3)
    return C.diag_heavy(n, N_GATES, SEED)


# kernel of each profiled op kind on the state (the profile counts each
# launch's algorithmic bytes: 2 x 2^n x bytes/amp for a read+write sweep,
# 2^n x bytes/amp for a write-only one)
KIND_KERNELS = {"chunk": "k_chunk (cache-blocked chunk sweep)", "diag": "k_diag (fused-diagonal sweep)",
                "dense": "k_dense5 (dense 5-qubit block)", "tensor": "k_tensor (merge-booster product)",
                "gate": "k_gate_dense (gate-by-gate)", "gate_diag": "k_gate_diag (gate-by-gate diagonal)"}


def _cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


REF_PREFIX_GATES = 64    # gates per reference-arm step (a bounded sample of the circuit)


def cpu_oracle_prefix(args, n_gates: int, threads: int):
    """Time the CPU oracle (complex128, gate by gate) on the first n_gates
    gates of the workload at min(n, 28) qubits, from its initial basis
    state; returns (seconds, gates run, qubits)."""
    import oracle
    n = min(N_QUBITS, 28)
    c = _workload_circuit(args, n)
    a = oracle.basis_state(n, c.basis)
    gl = c.gates[:n_gates]
    t0 = time.perf_counter()
    oracle.run_inplace(n, a, gl, threads)
    dt = time.perf_counter() - t0
    del a
    return dt, len(gl), n


def oracle_full_run(args, threads: int):
    """The whole workload circuit on the CPU oracle (complex128, gate by gate,
    Algorithm 1), timed: returns (state, seconds).  Only for workloads the
    host holds in full (n <= 28: 4 GiB)."""
    import oracle
    c = _workload_circuit(args, N_QUBITS)
    a = oracle.basis_state(N_QUBITS, c.basis)
    t0 = time.perf_counter()
    oracle.run_inplace(N_QUBITS, a, c.gates, threads)
    return a, time.perf_counter() - t0


def state_error(got, exp, step=1 << 24):
    """max |got - exp|, |<exp|got>|^2 / (<got|got><exp|exp>) and the norm of
    got, over slices (no full-size temporaries)."""
    import numpy as np
    err, ov, ng, ne = 0.0, 0j, 0.0, 0.0
    for lo in range(0, exp.size, step):
        g = got[lo:lo + step].astype(np.complex128)
        e = exp[lo:lo + step]
        err = max(err, float(np.max(np.abs(g - e))))
        ov += np.vdot(e, g)
        ng += float(np.vdot(g, g).real)
        ne += float(np.vdot(e, e).real)
    return err, float(abs(ov) ** 2 / (ng * ne)), ng


def error_without_oracle(args, sim, buf, circ, opt, dt):
    """The error of a final state too large for the host oracle.  QFT and the
    full-connectivity RZZ stream have closed forms (QFT|x> = 2^(-n/2)
    sum_y e^{2 pi i x y / 2^n} |y>; RZZ after H on every qubit: 2^(-n/2)
    exp(-i/2 sum_{a<b} theta_ab s_a s_b), s_q = 1 - 2 x_q), compared on 2^16
    seeded random indices and a run of 2^16; other circuits are followed by
    their inverse and the distance from the initial basis state is reported."""
    import numpy as np
    import torch
    from paper_2604_12256_gb300 import circuits as C
    from paper_2604_12256_gb300 import svsim as S
    n = circ.n
    rng = np.random.default_rng(7)
    idx = np.unique(np.concatenate([rng.integers(0, 1 << n, 1 << 16, dtype=np.int64),
                                    np.arange(1 << 20, (1 << 20) + (1 << 16), dtype=np.int64)]))
    if args.workload in ("qft", "rzz-full"):
        torch.cuda.synchronize()
        cv = buf.view(torch.complex128 if dt == S.SIM_C128 else torch.complex64)
        got = cv[torch.as_tensor(idx, device="cuda")].cpu().numpy().astype(np.complex128)
        amp = 2.0 ** (-n / 2)
        if args.workload == "qft":
            x = circ.basis
            ph = ((np.uint64(x) * idx.astype(np.uint64)) & np.uint64((1 << n) - 1)).astype(np.float64) / float(1 << n)
            exp = amp * np.exp(2j * np.pi * ph)
        else:
            theta = np.zeros((n, n))
            for g in circ.gates:
                if g.kind == "rzz":
                    theta[g.qubits[0], g.qubits[1]] += g.params[0]
            sgn = 1.0 - 2.0 * ((idx[:, None] >> np.arange(n)[None, :]) & 1).astype(np.float64)
            exp = amp * np.exp(-0.5j * np.einsum("ia,ab,ib->i", sgn, theta, sgn))
        err = float(np.max(np.abs(got - exp)))
        return {"vs": "closed form on %d sampled amplitudes" % idx.size, "state_max_abs": err,
                "state_max_rel": err / amp,
                "tolerance": {"state_max_abs": 1e-5 if dt == S.SIM_C64 else 1e-12}}
    inv = C.inverse(circ)
    sim.apply(inv.gates, opt)
    ti, tp = sim.top_k(2)
    return {"vs": "the inverse circuit applied after the circuit: distance from the initial basis state",
            "one_minus_p_initial": float(1.0 - tp[0]) if int(ti[0]) == circ.basis else 1.0,
            "largest_other_p": float(tp[1]), "norm": sim.norm()}


def run_reference(args, rank, world):
    """The oracle as it stands on the host cores.  One step = the first
    REF_PREFIX_GATES gates of the workload at min(n, 28) qubits (a bounded
    sample: the whole 528-gate circuit takes about half a minute on 16 cores,
    and the run has 25 steps); ms_per_step is that measured time."""
    if rank != 0:
        return
    cores = _cores()
    for _ in range(args.warmup):
        cpu_oracle_prefix(args, REF_PREFIX_GATES, cores)
    times = []
    for _ in range(args.steps):
        dt, g, n = cpu_oracle_prefix(args, REF_PREFIX_GATES, cores)
        times.append(dt)
    ms = 1e3 * statistics.median(times)
    v = g * (1 << n) / (ms / 1e3)
    G = len(_workload_circuit(args, N_QUBITS).gates)
    sample = (f"each step: gates 1..{g} of the {G}-gate workload circuit at {n} qubits from its initial basis "
              f"state, complex128, gate by gate on {cores} host threads; median of {args.steps} steps")
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_qubits": N_QUBITS, "gates": G,
                       "seed": SEED, "l2": "state larger than L2", "step": f"first {g} gates (bounded sample)"},
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args, rank, world, dist):
    import torch
    from paper_2604_12256_gb300 import build as B
    from paper_2604_12256_gb300 import svsim as S

    B.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    dense = args.workload == "layered-dense"
    dt = S.SIM_C128 if args.dtype == "c128" else S.SIM_C64
    s_amp = 16 if dt == S.SIM_C128 else 8
    circ = _workload_circuit(args, N_QUBITS)
    ga = S.GateArray(circ.gates)
    G = len(circ.gates)
    amps = 1 << N_QUBITS
    # the state lives in a torch-owned HBM buffer; kernels run on torch's stream
    buf = torch.empty(amps * s_amp // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    sim = S.Sim(N_QUBITS, dt, dev_buf=buf.data_ptr(), nbytes=buf.numel() * 4, stream=stream.cuda_stream)
    opt = S.default_options()
    if dense:
        # split-TF32 complex64 blocks run cache-blocked (several per sweep on
        # the tensor cores) unless --dense-separate asks for one sweep each
        opt.flags = S.SIM_F_TC | S.SIM_F_DIAG | (0 if args.dense_separate else S.SIM_F_BLOCK)
        opt.dense_precision = PRECISIONS[args.precision]
    fused_dense = dense and dt == S.SIM_C64 and args.precision == "tf32x3" and not args.dense_separate
    if args.register_bits:
        opt.register_bits = args.register_bits
    if args.chunk_qubits:
        opt.chunk_qubits = args.chunk_qubits
    if args.jit and not dense:
        # chunk sweeps run kernels specialised to their programs, compiled
        # (NVRTC) during the first warm-up step and cached
        opt.flags |= S.SIM_F_JIT
    if args.remap:
        opt.flags |= S.SIM_F_REMAP

    def step():
        sim.reset(circ.basis)
        sim.apply(ga, opt)

    # cold: the first apply of this circuit's structure in the process
    # (specialised kernels generated and compiled by NVRTC on the way)
    jit_before = S.jit_info()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step()
    torch.cuda.synchronize()
    first_apply_ms = (time.perf_counter() - t0) * 1e3
    jit_first = S.jit_info()
    for _ in range(max(0, args.warmup - 1)):
        step()
    torch.cuda.synchronize()
    plan = sim.stats()

    def barrier():
        if dist is not None:
            dist.barrier()

    clocks = Clocks(dev)
    clocks.start()
    time.sleep(0.3)
    # per-launch CUDA events around the launches on the state (the roofline's
    # kernel durations); none around the booster's small sub-state launches
    sim.profile_enable(True, state_only=True)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0 = S.kernel_launches()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    gpu_launches = S.kernel_launches() - k0
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    prof = sim.profile_read()
    sim.profile_enable(False)
    clk = clocks.stop()
    ms = max_over_ranks(ms, dist)
    jit = S.jit_info()

    # end-to-end through the C ABI: host gate list in, host results out
    pairs = [(i, (i * 7 + 3) % N_QUBITS) for i in range(16)]
    masks = [(1 << a) | (1 << b) for a, b in pairs]
    torch.cuda.synchronize()
    te = []
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        sim.reset(circ.basis)
        sim.apply(circ.gates, opt)      # marshal from the Python gate list each step
        idx, p, ev = sim.top_k_expectation(64, masks)   # both read-outs, concurrently, one sync
        te.append(time.perf_counter() - t0)
    e2e_s = statistics.median(te)
    # the fused path's final state, for the error against the oracle below
    final_state = sim.get_state() if rank == 0 and not args.no_cpu_baseline and N_QUBITS <= 28 else None
    # states the host oracle does not hold: closed forms on sampled
    # amplitudes, or the inverse circuit's return to the initial state
    big_error = None
    if rank == 0 and N_QUBITS > 28:
        big_error = error_without_oracle(args, sim, buf, circ, opt, dt)
    # fresh angles: the same circuit structure with every angle (and Haar
    # one-qubit matrix) drawn anew, end to end through the C ABI; with
    # specialised kernels keyed by structure no compile is expected
    fresh = [_redraw(circ, 1000 + i) for i in range(max(3, min(args.steps, 10)))]
    jit_f0 = S.jit_info()
    tf = []
    for fc in fresh:
        t0 = time.perf_counter()
        sim.reset(fc.basis)
        sim.apply(fc.gates, opt)
        sim.top_k_expectation(64, masks)
        tf.append(time.perf_counter() - t0)
    jit_f1 = S.jit_info()
    fresh_angles = {"ms_per_step": statistics.median(tf) * 1e3, "circuits": len(fresh),
                    "value": world * G * amps / statistics.median(tf), "unit": UNIT,
                    "compiles": jit_f1["compiles"] - jit_f0["compiles"]}
    h2d = prof["h2d_bytes"] // max(1, args.steps)
    d2h = 64 * 16 + 16 * 8

    unfused = None
    if not args.no_unfused:
        # the unfused gate-by-gate GPU path on the same circuit (one timed run)
        unf = S.default_options(flags=0)
        sim.reset(circ.basis)
        sim.apply(ga, unf)
        torch.cuda.synchronize()
        u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        u0.record(stream)
        sim.reset(circ.basis)
        sim.apply(ga, unf)
        u1.record(stream)
        torch.cuda.synchronize()
        unf_ms = u0.elapsed_time(u1)
        unfused = {"ms_per_step": unf_ms, "value": G * amps / (unf_ms / 1e3), "speedup_fused_vs_unfused": unf_ms / ms}

    # the oracle leg: the whole circuit on the host cores (timed), and the
    # error of the GPU state and read-outs against it (rank 0, states the
    # host holds in full)
    oracle_leg = None
    if final_state is not None:
        import numpy as np
        import oracle
        got, final_state = final_state, None
        cores = _cores()
        exp, t_all = oracle_full_run(args, cores)
        err, fid, ng = state_error(got, exp)
        ref_idx, ref_p = oracle.top_k(exp, 64)
        ref_zz = oracle.expectation_z(exp, masks)
        del got, exp
        t1, g1, n1 = cpu_oracle_prefix(args, 8, 1)
        oracle_leg = {
            "cpu_baseline": {"value": G * amps / t_all, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"the whole {G}-gate circuit at {N_QUBITS} qubits, complex128, gate by gate, "
                                       f"{t_all:.1f} s on {cores} host threads (timed once)",
                             "seconds": t_all,
                             "one_thread": {"value": g1 * (1 << n1) / t1, "unit": UNIT, "cores": 1,
                                            "sample": f"gates 1..{g1} at {n1} qubits on 1 thread, {t1:.1f} s"}},
            "error": {"vs": "CPU oracle (complex128, gate by gate), same circuit",
                      "state_max_abs": err, "fidelity": fid, "norm": ng,
                      "top64_set_equal": bool(set(idx.tolist()) == set(ref_idx.tolist())),
                      "top64_prob_max_abs": float(np.max(np.abs(np.sort(p) - np.sort(ref_p)))),
                      "zz16_max_abs": float(np.max(np.abs(np.asarray(ev) - ref_zz))),
                      "tolerance": {"state_max_abs": 1e-5, "fidelity": 1 - 1e-6}
                      if dt == S.SIM_C64 else {"state_max_abs": 1e-12}},
        }

    peak, peak_kind = _peaks()
    # the dominant kernel: the op kind with the most device time on the state
    kind = max(KIND_KERNELS, key=lambda k: prof[k]["ms"] if isinstance(prof.get(k), dict) else -1)
    kp = prof[kind]
    nl = max(1, kp["launches"])
    avg_ms = kp["ms"] / nl
    bytes_per_launch = kp["bytes"] / nl
    kname = KIND_KERNELS[kind]
    if kind == "dense":
        kname = "k_dense5_tc (dense 5-qubit block, tcgen05 split-TF32)" if args.precision == "tf32x3" \
            and dt == S.SIM_C64 else "k_dense5_fma (dense 5-qubit block, CUDA cores)"
    jit_on = kind in ("chunk", "diag") and bool(opt.flags & S.SIM_F_JIT) and dt == S.SIM_C64
    ksrc = {"chunk": ("chunk_dev.cuh",), "diag": ("chunk_dev.cuh",),
            "dense": ("k_dense5.cu",)}.get(kind, ("k_basic.cu",)) + (("jit.cpp",) if jit_on else ())
    src = b"".join(open(os.path.join(ROOT, "paper_2604_12256_gb300", "csrc", f), "rb").read() for f in ksrc)
    tpa = TRAFFIC_PER_AMP.get((args.workload, kind + ("-jit" if jit_on else ""), hashlib.sha256(src).hexdigest()))
    if jit_on:
        kname = ("svs_chunk_jit (cache-blocked chunk sweep specialised to its program)" if kind == "chunk" else
                 "svs_diag_jit (fused-diagonal sweep specialised to its program)")
    if (dense and (args.precision != "tf32x3" or fused_dense)) or args.dtype != "c64":
        tpa = None   # captured on complex64 (and the one-block-per-sweep tensor-core kernel) only
    traffic = tpa * amps if tpa is not None else None
    if kind == "dense" and dt == S.SIM_C128:
        # double-float on the FP32 pipe: per amplitude 2 components x 64 real
        # multiply-adds of 15 FP32 flops (a product, three FMAs, a two-sum and
        # two adds), plus the final quick two-sums
        kname = "k_dense5_df (dense 5-qubit block, double-float on the FP32 pipe)"
        achieved = DF_FLOPS_PER_AMP * amps / (avg_ms / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}
    elif kind == "dense" and args.precision != "tf32x3":
        # 32 complex multiply-adds per amplitude: 256 real flops
        achieved = 256.0 * amps / (avg_ms / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}
    elif kind == "chunk" and dt == S.SIM_C128:
        # double-float chunk sweeps are bound by FP32 issue, not HBM: the plan's
        # flops (8 per complex multiply-add of a gate, 6 per phase product) at
        # 7.5 FP32 operations each (a double-float multiply-add issues about 15)
        achieved = plan["flops"] * DF_OPS_PER_FLOP * args.steps / (kp["ms"] / 1e3) / 1e12
        gbs = bytes_per_launch / (avg_ms / 1e3) / 1e9
        roof = {"bound": "alu", "kernel": kname + ", double-float", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
                "flop_per_amp": plan["flops"] / amps, "fp32_ops_per_flop": DF_OPS_PER_FLOP,
                "hbm": {"achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak}}
    elif kind == "dense" and fused_dense:
        # several blocks per sweep: the tensor pipe (three TF32 products of
        # 64 x 64 per 32 amplitudes and block) against the HBM round trip
        kname = "k_dense_chunk_tc (dense 5-qubit blocks inside the cache-blocked sweep, tcgen05 split-TF32)"
        tpeak, tsrc = _tf32_peak(sustained=True)
        tflops = TF32_FLOPS_PER_AMP_BLOCK * amps * plan["dense_ops"] * args.steps / (kp["ms"] / 1e3) / 1e12
        gbs = bytes_per_launch / (avg_ms / 1e3) / 1e9
        tc = {"achieved": tflops, "peak": tpeak, "unit": "TFLOP/s", "frac": tflops / tpeak, "peak_source": tsrc,
              "flop_per_amp_per_block": TF32_FLOPS_PER_AMP_BLOCK,
              "blocks_per_sweep": plan["dense_ops"] / max(1, plan["sweeps"])}
        hb = {"achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak, "peak_source": peak_kind}
        main = tc if tc["frac"] >= hb["frac"] else hb
        roof = {"bound": "tensor" if main is tc else "hbm", "kernel": kname, **main, "traffic": traffic,
                "tensor": tc, "hbm": hb}
    else:
        achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9 if kp["ms"] > 0 else None
        roof = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic, "peak_source": peak_kind}
    roof.update({"launches": kp["launches"], "avg_launch_ms": avg_ms, "algorithmic_bytes_per_launch": bytes_per_launch})
    total_bytes = sum(v["bytes"] for k, v in prof.items() if isinstance(v, dict)) / args.steps
    value = whole_job_rate(G * amps, world, ms / 1e3)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_qubits": N_QUBITS, "gates": G,
                       "seed": {"layered-dense": 0, "layered": 0, "rzz-full": 5, "qft": 2, "qaoa": 3}.get(args.workload, SEED),
                       "parallelism": f"replicas x{world}",
                       "l2": f"state ({amps * s_amp / 2 ** 30:g} GiB) larger than L2, no flush",
                       "sweeps": plan["sweeps"], "chunk_ops": plan["chunk_ops"], "dense_ops": plan["dense_ops"],
                       "diag_fused": plan["diag_fused"], "plan_ms": plan["plan_ms"],
                       **({"remap": True} if args.remap else {}),
                       "chunk_kernels": ("specialised per program structure at run time (NVRTC; numbers in the "
                                         "launch's parameter block), compiled in the first warm-up step and "
                                         "cached: %d kernels, %d compiles, %.0f ms of compile"
                                         % (jit["programs"], jit["compiles"], jit["compile_ms"]))
                       if opt.flags & S.SIM_F_JIT else "interpreter"},
            "hbm_gbs": total_bytes / (ms / 1e3) / 1e9,
            "hbm_frac_of_" + peak_kind: total_bytes / (ms / 1e3) / 1e9 / peak,
            "roofline": roof,
            "unfused": unfused,
            "e2e": {"value": world * G * amps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3,
                    "first_apply_ms": first_apply_ms,
                    "first_apply_compiles": jit_first["compiles"] - jit_before["compiles"],
                    "fresh_angles": fresh_angles},
            "gpu_launches": int(gpu_launches),
            "clocks": clk,
        }
        if oracle_leg is not None:
            line["cpu_baseline"] = oracle_leg["cpu_baseline"]
            line["error"] = oracle_leg["error"]
        elif big_error is not None:
            line["error"] = big_error
        print(json.dumps(line), flush=True)
    sim.close()


def run_families(args, rank, world, dist):
    """Per-gate time of the circuit families of Table 2 (BV, HS, QV, SC, VC)
    at one qubit count: gate by gate (no optimizer), optimized without the
    merge booster, and with it.  CUDA events on the handle's stream, median
    of --steps runs after --warmup."""
    import torch
    from paper_2604_12256_gb300 import build as B
    from paper_2604_12256_gb300 import circuits as C
    from paper_2604_12256_gb300 import svsim as S

    B.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    n = args.qubits or 28
    buf = torch.empty(2 << n, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    sim = S.Sim(n, S.SIM_C64, dev_buf=buf.data_ptr(), nbytes=buf.numel() * 4, stream=stream.cuda_stream)
    # interpreter kernels, then the kernels specialised to each sweep's
    # structure (compiled in the warm-up runs)
    configs = {"naive": S.default_options(flags=0),
               "ours": S.default_options(flags=S.SIM_F_DIAG | S.SIM_F_BLOCK | S.SIM_F_FUSE),
               "ours_b": S.default_options(),
               "ours_jit": S.default_options(flags=S.SIM_F_DIAG | S.SIM_F_BLOCK | S.SIM_F_FUSE | S.SIM_F_JIT),
               "ours_b_jit": S.default_options(flags=S.default_options().flags | S.SIM_F_JIT)}
    clocks = Clocks(dev)
    clocks.start()
    out = {}
    for fam, gen in sorted(C.FAMILIES.items()):
        c = gen(n if fam != "hs" or n % 2 == 0 else n - 1)
        ga = S.GateArray(c.gates)
        row = {"gates": len(c.gates)}
        for key, opt in configs.items():
            def step():
                sim.reset(c.basis)
                sim.apply(ga, opt)
            for _ in range(args.warmup):
                step()
            times = []
            for _ in range(args.steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step()
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            ms = statistics.median(times)
            st = sim.stats()
            row[key] = {"ms": ms, "ms_per_gate": ms / len(c.gates), "sweeps": st["sweeps"], "ops": st["ops"]}
        row["speedup_ours_vs_naive"] = row["naive"]["ms"] / row["ours"]["ms"]
        row["speedup_booster"] = row["ours"]["ms"] / row["ours_b"]["ms"]
        row["speedup_booster_jit"] = row["ours_jit"]["ms"] / row["ours_b_jit"]["ms"]
        row["speedup_jit_vs_naive"] = row["naive"]["ms"] / row["ours_b_jit"]["ms"]
        out[fam] = row
    clk = clocks.stop()
    sim.close()
    if rank == 0:
        line = {"metric": "per-gate time of the circuit families (Table 2)", "unit": "ms/gate", "n_qubits": n,
                "dtype": "c64", "data": "synthetic", "steps": args.steps, "warmup": args.warmup,
                "higher_is_better": False, "families": out, "clocks": clk}
        print(json.dumps(line), flush=True)


def run_readouts(args, rank, world, dist):
    """Time of the read-outs (K9) on the workload's final state: top-64, the
    sixteen <Z_a Z_b> of the e2e leg, and the norm.  Each call returns its
    result in host memory, so it ends with a synchronise and a small copy;
    the CUDA-event time of a call (the handle's stream) counts its kernels
    and that copy, the wall time the host side too.  Median of --steps calls
    after --warmup.  Each read-out reads the state once: 2^n x 8 bytes."""
    import torch
    from paper_2604_12256_gb300 import build as B
    from paper_2604_12256_gb300 import svsim as S

    B.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    n = args.qubits or N_QUBITS
    circ = _workload_circuit(args, n)
    buf = torch.empty(2 << n, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    sim = S.Sim(n, S.SIM_C64, dev_buf=buf.data_ptr(), nbytes=buf.numel() * 4, stream=stream.cuda_stream)
    opt = S.default_options()
    if args.jit:
        opt.flags |= S.SIM_F_JIT
    sim.reset(circ.basis)
    sim.apply(circ.gates, opt)
    torch.cuda.synchronize()
    masks = [(1 << a) | (1 << ((a * 7 + 3) % n)) for a in range(16)]
    calls = {"top64": lambda: sim.top_k(64), "zz16": lambda: sim.expectation(masks), "norm": lambda: sim.norm(),
             "top64+zz16 (one call, concurrent)": lambda: sim.top_k_expectation(64, masks)}
    peak, peak_kind = _peaks()
    state_bytes = (1 << n) * 8
    clocks = Clocks(dev)
    clocks.start()
    out = {}
    for name, call in calls.items():
        for _ in range(args.warmup):
            call()
        ev, wall = [], []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            e0.record(stream)
            call()
            e1.record(stream)
            torch.cuda.synchronize()
            wall.append((time.perf_counter() - t0) * 1e3)
            ev.append(e0.elapsed_time(e1))
        ms = statistics.median(ev)
        gbs = state_bytes / (ms / 1e3) / 1e9
        out[name] = {"ms": ms, "wall_ms": statistics.median(wall), "hbm_gbs": gbs,
                     "hbm_frac_of_" + peak_kind: gbs / peak}
    clk = clocks.stop()
    sim.close()
    if rank == 0:
        line = {"metric": "read-out time per call (top-64, 16 <ZZ>, norm)", "unit": "ms", "n_qubits": n,
                "dtype": "c64", "data": "synthetic", "workload": args.workload, "steps": args.steps,
                "warmup": args.warmup, "higher_is_better": False, "bytes_per_call": state_bytes,
                "readouts": out, "clocks": clk}
        print(json.dumps(line), flush=True)


FP64_PEAK_TFLOPS = 1.25    # nominal dense FP64 of a GB300 (no measured figure on this machine)


def run_precision(args, rank, world, dist):
    """Config 3's precision study: the depth-20 random layered circuit fused
    into dense 5-qubit blocks, run in every arithmetic arm, each timed (CUDA
    events around the whole apply, one run after a smaller warm-up circuit)
    and compared with a complex128 GPU reference state on the device: true
    FP64 blocks at n <= 30, double-float above (the FP64 run grows to minutes
    there; double-float agrees with it to about 1e-14, tests/test_gpu_dense).
    Both reference arms are checked against the CPU oracle at <= 24 qubits by
    the GPU tests.  Error = max |a - a_ref| and |<a_ref|a>|^2 / norms, in FP64
    over slices of the states (no full-size temporaries)."""
    import torch
    from paper_2604_12256_gb300 import build as B
    from paper_2604_12256_gb300 import circuits as C
    from paper_2604_12256_gb300 import svsim as S

    B.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    n = args.qubits or 33
    circ = C.layered(n, 20, 0)
    ga = S.GateArray(circ.gates)
    warm = S.GateArray(C.layered(n, 1, 1).gates)
    stream = torch.cuda.current_stream()
    amps = 1 << n
    ref_prec = "fp64" if n <= 30 else "double-float"
    # (dtype, arithmetic, cache-blocked block sweeps): split-TF32 both ways
    arms = [("c128", ref_prec, False)] + [("c128", "double-float", False)] * (ref_prec == "fp64") + \
           [("c64", "tf32x3", True), ("c64", "tf32x3", False), ("c64", "fp32", False)]
    code = {"tf32x3": S.SIM_DENSE_SPLIT_TF32, "fp32": S.SIM_DENSE_FP32, "fp64": S.SIM_DENSE_FP64,
            "double-float": S.SIM_DENSE_DOUBLE_FLOAT}
    clocks = Clocks(dev)
    clocks.start()
    ref = None
    out = []
    for dt_name, prec, blocked in arms:
        c128 = dt_name == "c128"
        buf = torch.empty(2 * amps, dtype=torch.float64 if c128 else torch.float32, device="cuda")
        sim = S.Sim(n, S.SIM_C128 if c128 else S.SIM_C64, dev_buf=buf.data_ptr(),
                    nbytes=buf.numel() * buf.element_size(), stream=stream.cuda_stream)
        opt = S.default_options(flags=S.SIM_F_TC | S.SIM_F_DIAG | (S.SIM_F_BLOCK if blocked else 0),
                                dense_precision=code[prec])
        sim.reset(0)
        sim.apply(warm, opt)
        sim.profile_enable(True, state_only=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.reset(0)
        sim.apply(ga, opt)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        prof = sim.profile_read()
        st = sim.stats()
        sim.close()
        cv = buf.view(torch.complex128 if c128 else torch.complex64)
        d = prof["dense"]
        sweep_ms = d["ms"] / max(1, d["launches"])
        if prec == "tf32x3" and blocked:
            tpeak, tsrc = _tf32_peak(sustained=True)
            roof = {"bound": "tensor",
                    "achieved": TF32_FLOPS_PER_AMP_BLOCK * amps * st["dense_ops"] / (d["ms"] / 1e3) / 1e12,
                    "peak": tpeak, "unit": "TFLOP/s", "peak_source": tsrc, "kernel": "k_dense_chunk_tc",
                    "flop_per_amp_per_block": TF32_FLOPS_PER_AMP_BLOCK,
                    "hbm_frac": 16.0 * amps / (sweep_ms / 1e3) / 1e9 / _peaks()[0]}
        elif prec == "tf32x3":
            roof = {"bound": "hbm", "achieved": 16.0 * amps / (sweep_ms / 1e3) / 1e9, "peak": _peaks()[0],
                    "unit": "GB/s", "kernel": "k_dense5_tc"}
        elif prec == "fp32":
            roof = {"bound": "alu", "achieved": 256.0 * amps / (sweep_ms / 1e3) / 1e12, "peak": FP32_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "kernel": "k_dense5_fma<float>",
                    "flop_per_amp": 256, "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}
        elif prec == "double-float":
            roof = {"bound": "alu", "achieved": DF_FLOPS_PER_AMP * amps / (sweep_ms / 1e3) / 1e12,
                    "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "kernel": "k_dense5_df",
                    "flop_per_amp": DF_FLOPS_PER_AMP,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz (FP32 operations of the "
                                   "double-float arithmetic)"}
        else:
            roof = {"bound": "alu", "achieved": 256.0 * amps / (sweep_ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "kernel": "k_dense5_fma<double>", "flop_per_amp": 256,
                    "peak_source": "nominal FP64 of a GB300"}
        roof["frac"] = roof["achieved"] / roof["peak"]
        row = {"dtype": dt_name, "arith": prec, "ms": ms, "blocks": st["dense_ops"], "sweeps": st["sweeps"],
               "cache_blocked": blocked, "ms_per_sweep": sweep_ms,
               "amplitude_updates_per_s": len(circ.gates) * amps / (ms / 1e3), "roofline": roof}
        if ref is None:
            ref, ref_buf = cv, buf
            row["error"] = "reference"
        else:
            err, ov, ng, ne = 0.0, 0j, 0.0, 0.0
            step = 1 << 26
            for lo in range(0, amps, step):
                a = cv[lo:lo + step].to(torch.complex128)
                r = ref[lo:lo + step]
                err = max(err, float((a - r).abs().max()))
                ov += complex(torch.vdot(r, a))
                ng += float(torch.vdot(a, a).real)
                ne += float(torch.vdot(r, r).real)
            row["error"] = {"max_abs": err, "fidelity": abs(ov) ** 2 / (ng * ne), "norm": ng,
                            "vs": f"complex128 {ref_prec} GPU state"}
            del cv, buf
            torch.cuda.empty_cache()
        out.append(row)
    clk = clocks.stop()
    if rank == 0:
        line = {"metric": "precision study: time, roofline and error of the dense 5-qubit block arms (config 3)",
                "n_qubits": n, "workload": f"{n}-qubit random layered circuit, depth 20, dense 5-qubit blocks",
                "gates": len(circ.gates), "data": "synthetic", "reference": f"complex128 {ref_prec} on the GPU",
                "arms": out, "clocks": clk}
        print(json.dumps(line), flush=True)


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(round(q * (len(xs) - 1))))] if xs else None


def run_serve(args, rank, world, dist):
    """Serving stream: requests of 10-26 qubits, depth 10-200, families
    layered / diagonal-heavy / QFT / QAOA, each returning the top-64
    probabilities and 16 <Z_i Z_j>, complex64.  Measured: the serial
    one-circuit-at-a-time capacity through sim_* handles, then the server
    (srv_*: continuous batching, admission by state footprint) under Poisson
    arrivals at 0.5 / 0.8 / 1.2 x that capacity and with every request
    queued at once (saturated).  Gate lists are marshalled before timing."""
    import numpy as np
    import torch
    from paper_2604_12256_gb300 import build as B
    from paper_2604_12256_gb300 import circuits as C
    from paper_2604_12256_gb300 import svsim as S

    B.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    R = args.requests
    reqs = C.serving_stream(R, 1.0, seed=4 + rank)          # unit-rate arrivals, rescaled below
    arr1 = [r.arrival_s for r in reqs]
    gas = [S.GateArray(r.circuit.gates) for r in reqs]
    masks = [[int(m) for m in C.z_masks(r.z_pairs)] for r in reqs]
    h2d = sum(g.n for g in gas) * ctypes_sizeof_gate(S) / R
    d2h = 64 * 16 + 16 * 8

    def barrier():
        if dist is not None:
            dist.barrier()

    # serial capacity: one handle per qubit count, one request at a time
    sims = {}
    for n in sorted({r.circuit.n for r in reqs}):
        sims[n] = S.Sim(n, S.SIM_C64)
    ser = [None] * R

    def serial(i):
        r = reqs[i]
        sm = sims[r.circuit.n]
        sm.reset(r.circuit.basis)
        sm.apply(gas[i])
        idx, p = sm.top_k(64)
        ser[i] = (idx, p, sm.expectation(masks[i]))

    for i in range(min(R, 32)):
        serial(i)
    torch.cuda.synchronize()
    clocks = Clocks(dev)
    clocks.start()
    time.sleep(0.3)
    barrier()
    k0 = S.kernel_launches()
    t0 = time.perf_counter()
    svc = []
    for i in range(R):
        a = time.perf_counter()
        serial(i)
        svc.append((time.perf_counter() - a) * 1e3)
    serial_s = time.perf_counter() - t0
    serial_launches = S.kernel_launches() - k0
    serial_cps = R / serial_s
    for sm in sims.values():
        sm.close()

    budget = int(args.budget_gib * (1 << 30))

    def serve(rate_hz):
        """rate_hz None: everything queued at t = 0."""
        with S.Server(budget, n_streams=args.streams) as srv:
            tk = [0] * R
            k0 = S.kernel_launches()
            t0 = time.perf_counter()
            for i in range(R):
                if rate_hz is not None:
                    wait = t0 + arr1[i] / rate_hz - time.perf_counter()
                    if wait > 0:
                        time.sleep(wait)
                tk[i] = srv.submit_array(gas[i], reqs[i].circuit.n, reqs[i].circuit.basis, 64, masks[i])
            res = [srv.poll(t) for t in tk]
            wall = time.perf_counter() - t0
            st = srv.stats()
            kl = S.kernel_launches() - k0
        dexp = max(float(np.max(np.abs(r["expect"] - ser[i][2]))) for i, r in enumerate(res))
        dp = max(float(np.max(np.abs(r["top_p"] - ser[i][1]))) for i, r in enumerate(res))
        return {"offered_hz": rate_hz, "circuits_per_s": R / wall, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                "mean_ms": st["mean_ms"], "max_ms": st["max_ms"], "failed": int(st["failed"]),
                "batched": int(st["batched"]), "batch_launches": int(st["batches"]),
                "hbm_peak_gib": st["hbm_peak"] / 2 ** 30, "kernel_launches": int(kl),
                "max_abs_diff_vs_serial": {"expect": dexp, "top_p": dp}}

    sat = serve(None)
    pois = []
    for f in (0.5, 0.8, 1.2):
        d = serve(f * serial_cps)
        d["load"] = f
        pois.append(d)
    clk = clocks.stop()
    value = whole_job_rate(R, world, max_over_ranks(R / sat["circuits_per_s"], dist))
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "circuits/s", "n_gpus": world, "steps": R,
            "warmup": min(R, 32), "ms_per_step": 1e3 / sat["circuits_per_s"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": f"serving stream: {R} requests, qubits uniform 10-26, depth uniform 10-200, "
                                   "family uniform over layered / diagonal-heavy / QFT / QAOA, top-64 "
                                   "probabilities + 16 <Z_i Z_j> each, complex64",
                       "requests": R, "worker_streams": args.streams, "hbm_budget_gib": args.budget_gib,
                       "parallelism": f"replicas x{world}",
                       "l2": "states up to 512 MiB; no flush (requests run back to back as in service)"},
            "saturated": sat,
            "poisson": pois,
            "serial": {"circuits_per_s": serial_cps, "p50_ms": _pct(svc, 0.5), "p99_ms": _pct(svc, 0.99),
                       "kernel_launches": int(serial_launches),
                       "note": "one request at a time through sim_* handles (one per qubit count); "
                               "latency = service time, no queueing"},
            "speedup_vs_serial": value / world / serial_cps,
            "e2e": {"value": value, "unit": "circuits/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(sat["kernel_launches"]),
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)


def ctypes_sizeof_gate(S):
    import ctypes
    return ctypes.sizeof(S.sim_gate)


def main():
    global N_QUBITS, WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--register-bits", type=int, default=0,
                    help="chunk bits per thread in the cache-blocked kernel (0 = library default)")
    ap.add_argument("--chunk-qubits", type=int, default=0,
                    help="qubits per cached chunk (0 = library default)")
    ap.add_argument("--workload", default="diag-heavy",
                    choices=["diag-heavy", "layered-dense", "layered", "rzz-full", "qft", "qaoa"],
                    help="diag-heavy: the 28-qubit gate-level stream; layered-dense: depth-20 layered "
                         "circuit in dense 5-qubit blocks; layered: the same circuit on the default "
                         "cache-blocked path; rzz-full: RZZ on every qubit pair from |+...+> "
                         "(the last three: 34 qubits complex64 / 33 complex128 by default); qft, qaoa: "
                         "the 30-qubit circuit-level pair (QFT with the reversal SWAPs on a random basis "
                         "state; QAOA p = 4 on a random 3-regular graph)")
    ap.add_argument("--dense-separate", action="store_true",
                    help="layered-dense: one sweep per dense block instead of cache-blocked block sweeps")
    ap.add_argument("--precision", default="tf32x3", choices=sorted(PRECISIONS),
                    help="dense-block arithmetic for --workload layered-dense")
    ap.add_argument("--dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--no-jit", dest="jit", action="store_false",
                    help="run the chunk sweeps on the interpreter kernel instead of kernels specialised to "
                         "their programs")
    ap.add_argument("--no-unfused", action="store_true", help="skip the gate-by-gate comparison run")
    ap.add_argument("--readouts", action="store_true",
                    help="time the read-outs (top-64, 16 <ZZ>, norm) on the workload's final state")
    ap.add_argument("--remap", action="store_true",
                    help="persistent qubit frame: each block's store moves the qubits later blocks need into "
                         "the low positions")
    ap.add_argument("--families", action="store_true",
                    help="per-gate time of the BV / HS / QV / SC / VC families: gate by gate, optimized, "
                         "optimized with the merge booster")
    ap.add_argument("--precision-study", action="store_true",
                    help="config 3: the layered circuit in dense 5-qubit blocks in every arithmetic arm (split-TF32, "
                         "FP32, double-float, FP64), each timed and compared with a complex128 GPU reference")
    ap.add_argument("--serve", action="store_true",
                    help="time the serving loop on a Poisson request stream instead")
    ap.add_argument("--requests", type=int, default=10000, help="serving requests (config 4: 10,000)")
    ap.add_argument("--streams", type=int, default=4, help="serving worker streams")
    ap.add_argument("--budget-gib", type=float, default=32.0, help="serving HBM budget for admitted states")
    ap.add_argument("--qubits", type=int, default=0,
                    help="qubits of the workload (0: its default; smaller for ncu captures)")
    args = ap.parse_args()
    if args.workload == "layered":
        n = args.qubits or (33 if args.dtype == "c128" else 34)
        WORKLOAD = (f"{n}-qubit random layered circuit, depth 20 (Haar U(2) on every qubit, CZ brickwork), "
                    f"cache-blocked path, {'complex128' if args.dtype == 'c128' else 'complex64'}")
        N_QUBITS = n
    elif args.workload == "layered-dense":
        n = args.qubits or (33 if args.dtype == "c128" else 34)
        WORKLOAD = (f"{n}-qubit random layered circuit, depth 20 (Haar U(2) on every qubit, CZ brickwork), "
                    f"fused into dense 5-qubit blocks ({args.precision if args.dtype == 'c64' else 'double-float'}), "
                    f"{'complex128' if args.dtype == 'c128' else 'complex64'}")
        N_QUBITS = n
    elif args.workload == "rzz-full":
        n = args.qubits or (33 if args.dtype == "c128" else 34)
        WORKLOAD = (f"{n}-qubit full-connectivity RZZ gate-level stream ({n * (n - 1) // 2} RZZ, angles uniform "
                    f"in [0, 2pi), after H on every qubit), {'complex128' if args.dtype == 'c128' else 'complex64'}")
        N_QUBITS = n
    elif args.workload in ("qft", "qaoa"):
        n = args.qubits or 30
        WORKLOAD = (f"{n}-qubit QFT (H + controlled-phase ladder + reversal SWAPs) on a random basis state"
                    if args.workload == "qft" else
                    f"{n}-qubit QAOA p = 4 on a random 3-regular graph (RZZ per edge, RX mixer)")
        WORKLOAD += f", {'complex128' if args.dtype == 'c128' else 'complex64'}"
        N_QUBITS = n
    elif args.qubits and args.qubits != N_QUBITS:
        WORKLOAD = WORKLOAD.replace(f"{N_QUBITS}-qubit", f"{args.qubits}-qubit")
        N_QUBITS = args.qubits
    if args.dtype == "c128" and args.workload == "diag-heavy":
        WORKLOAD = WORKLOAD.replace("complex64", "complex128")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist_.init_process_group("nccl")
        dist = dist_
    try:
        (run_serve if args.serve else run_families if args.families else run_readouts if args.readouts
         else run_precision if args.precision_study else run_gpu)(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
