"""Benchmark: Wiener inverse PFB + up-channelization on one B300 (or N replicas).

Workload (the large single-stream configuration): lblock 4096, ntap 4, sinc x
Hamming window, 65536 spectra (2^28 samples), Gaussian noise plus 16 random
tones (seed 2), FP32 on the GPU, 4-bit quantized spectra with per-channel step
RMS/2.5; Wiener inversion with phi^2 measured from the simulation, then
up-channelization by 64 (real FFTs of 262144 samples over consecutive blocks).

One step = one call of ipfb_wiener_upchannelize over the resident 4-bit codes
(unpack + per-frame inverse FFT, per-column frame-axis FFT + Wiener gain +
inverse FFT, block real FFT).  The forward PFB that simulates the codes runs
before timing and is reported separately under "stages".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank inverts its own stream (replicas, no data-path
collective; weak scaling); rank 0 prints one JSON line.
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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LBLOCK, NTAP, NFRAMES, UPFACTOR = 4096, 4, 65536, 64
NSAMP = LBLOCK * NFRAMES
METRIC = "iPFB GSa/s at lblock=4096 ntap=4"
UNIT = "GSa/s"
WORKLOAD = "wiener_ipfb+upchannelize lblock=4096 ntap=4 nframes=65536 upfactor=64 (2^28 samples)"

KERNEL_FILES = {
    "k2_unpack_irfft": ["ipfb_kernels.cuh", "common.cuh", "k2_unpack.cu"],
    "k3_column_wiener": ["ipfb_kernels.cuh", "common.cuh", "k3_launch.cuh", "k3_cl_nt4.cu"],
    "k4_upchan": ["upchan_kernels.cuh", "common.cuh", "k4_upchan.cu"],
    "k4a_upchan_frames": ["upchan2_kernels.cuh", "common.cuh", "k4ab_upchan.cu"],
    "k4b_upchan_pairs": ["upchan2_kernels.cuh", "common.cuh", "k4ab_upchan.cu"],
    "k1_pfb_power": ["pfb_kernels.cuh", "common.cuh", "k1_forward.cu"],
    "k1_pfb_quant": ["pfb_kernels.cuh", "common.cuh", "k1_forward.cu"],
}


def kernel_source_hash(name: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_FILES.get(name, []):
        with open(os.path.join(ROOT, "paper_2608_23441_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def ncu_traffic(name: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current source of that kernel (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(name)
    if not d or d.get("source_hash") != kernel_source_hash(name):
        return None
    return float(d["dram_bytes_per_launch_full_size"])


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """SM clock and clock-event reasons during the timed region: the driver's NVML
    polled every 5 ms from a background thread (read-only queries), with an
    nvidia-smi -lms 200 sampler beside it as a fallback."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASON_BITS = {"hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
                   "sw_power_cap": 0x4, "hw_power_brake_slowdown": 0x80}

    def __init__(self, gpu_index: int, pci_bus_id: str | None = None):
        self.idx = gpu_index
        self.pci = pci_bus_id
        self.proc = None
        self.path = os.path.join("/tmp", f"ipfb_clocks_{os.getpid()}.csv")
        self.nv = []          # (sm_mhz, max_mhz, reasons bitmask)
        self.nv_err = None
        self._stop = None
        self._thr = None

    @staticmethod
    def _nvml():
        """The driver's NVML library through ctypes (read-only queries only)."""
        import ctypes
        for name in ("libnvidia-ml.so.1", "libnvidia-ml.so"):
            try:
                return ctypes.CDLL(name)
            except OSError:
                pass
        raise OSError("libnvidia-ml not found")

    def _nvml_loop(self):
        import ctypes
        try:
            nv = self._nvml()
            if nv.nvmlInit_v2() != 0:
                raise RuntimeError("nvmlInit failed")
            h = ctypes.c_void_p()
            ok = self.pci is not None and nv.nvmlDeviceGetHandleByPciBusId_v2(self.pci.encode(), ctypes.byref(h)) == 0
            if not ok and nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.idx), ctypes.byref(h)) != 0:
                raise RuntimeError("no NVML handle")
            NVML_CLOCK_SM = 1
            mx, sm, rs = ctypes.c_uint(0), ctypes.c_uint(0), ctypes.c_ulonglong(0)
            nv.nvmlDeviceGetMaxClockInfo(h, NVML_CLOCK_SM, ctypes.byref(mx))
            get_rs = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons
            while not self._stop.is_set():
                if nv.nvmlDeviceGetClockInfo(h, NVML_CLOCK_SM, ctypes.byref(sm)) == 0 and \
                        get_rs(h, ctypes.byref(rs)) == 0:
                    self.nv.append((sm.value, mx.value, rs.value))
                self._stop.wait(0.005)
            nv.nvmlShutdown()
        except Exception as e:  # reported in the summary; the nvidia-smi samples remain
            self.nv_err = f"{type(e).__name__}: {e}"[:160]

    def __enter__(self):
        import threading
        self._stop = threading.Event()
        self._thr = threading.Thread(target=self._nvml_loop, daemon=True)
        self._thr.start()
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self._stop is not None:
            self._stop.set()
            self._thr.join(timeout=5)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.nv:
            sm = [x[0] for x in self.nv]
            reasons = sorted({nm for _, _, rs in self.nv for nm, bit in self.REASON_BITS.items() if rs & bit})
            return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(x[1] for x in self.nv), "reasons": reasons,
                    "samples": len(sm), "source": "nvml, 5 ms"}
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "nvml_error": self.nv_err}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvidia-smi, 200 ms", "nvml_error": self.nv_err}


# --------------------------------------------------------------------------- distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(ws, backend: str = "nccl"):
    """One process per GPU (torchrun env); the replicas share nothing but the timing
    reduction.  backend "gloo" runs the same host logic on CPU ranks."""
    if ws <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group(backend=backend)
    return dist


def barrier(dist, torch):
    if dist is not None:
        dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()


def max_over_ranks(dist, torch, v: float) -> float:
    """The slowest rank's time: the job is done when every replica is."""
    if dist is None:
        return v
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gsas(ws: int, ms_max: float) -> float:
    """Whole-job throughput: every rank inverts its own 2^28-sample batch (weak
    scaling), divided by the slowest rank's time per step."""
    return ws * NSAMP / (ms_max * 1e-3) / 1e9


# --------------------------------------------------------------------------- CPU baseline
ORACLE_SAMPLE_FRAMES = 8192


def oracle_sample_step(codes, scale, window, phi2):
    """The FP64 oracle on one bounded sample of the workload: the same lblock,
    window and up-channelization factor, 8192 spectra (2^25 samples)."""
    from oracle import ipfb as oipfb
    from oracle import upchan as oup
    x = oipfb.ipfb_wiener(codes, scale, window, phi2)
    return oup.upchannelize(x, UPFACTOR * LBLOCK)


def oracle_sample_inputs():
    from oracle import pfb as opfb
    from paper_2608_23441_b300 import synth
    x = synth.stream_config(LBLOCK, ORACLE_SAMPLE_FRAMES, 2, ntones=16)
    w = opfb.sinc_hamming_window(LBLOCK, NTAP).astype(np.float32).astype(np.float64)
    codes, scale, spec = opfb.pfb_forward(x, w)
    phi2 = float(np.var(opfb.dequantize(codes, scale) - spec) / np.var(spec))
    return codes, scale, w, phi2


def cpu_baseline_measure(steps: int = 1, allcores: bool = True):
    """The oracle on a bounded sample of the workload: single-threaded, and on every
    host core at once (one sample per process); `value` is the all-core figure."""
    inp = oracle_sample_inputs()
    ts = []
    for _ in range(max(1, steps)):
        t0 = time.perf_counter()
        oracle_sample_step(*inp)
        ts.append(time.perf_counter() - t0)
    del inp
    sec = statistics.median(ts)
    single = ORACLE_SAMPLE_FRAMES * LBLOCK / sec / 1e9
    out = {"value": single, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{ORACLE_SAMPLE_FRAMES} spectra x lblock {LBLOCK} (2^25 samples) of the same workload, "
                     f"FP64 numpy oracle, single-threaded pocketfft, median of {len(ts)}",
           "seconds_per_sample": sec, "single_core": {"value": single, "cores": 1}, "nproc": host_cores()}
    if allcores:
        ac = cpu_baseline_allcores()
        out.update({"value": ac["value"], "cores": ac["procs"],
                    "all_cores": {"value": ac["value"], "cores": ac["procs"], "wall_s": ac["walls"][0],
                                  "host_cores": ac["host_cores"]},
                    "sample": out["sample"] + f"; all cores: {ac['procs']} single-threaded processes of "
                              f"{ac['host_cores']} host cores, one such sample each"})
    return out


def _oracle_worker(barrier, results, nsteps):
    """One host process of the all-core baseline: build the sample (untimed), then for
    every step wait for all processes and time one oracle step on the shared wall clock."""
    inp = oracle_sample_inputs()
    for i in range(nsteps):
        barrier.wait()
        t0 = time.time()
        oracle_sample_step(*inp)
        results.put((i, t0, time.time()))


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def host_mem_available_gb() -> float:
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 8.0


def cpu_baseline_allcores(nsteps: int = 1, timeout_s: float = 900.0):
    """The oracle, unchanged, on every host core at once: one process per core (spawned,
    so no process forks after the GPU is in use; each single-threaded), each inverting
    and up-channelizing its own 2^25-sample sample of the workload, `nsteps` times;
    per step, throughput = the samples of all processes / the wall time from the first
    start to the last finish.  The process count is capped by host memory (about 3 GB
    per process) and 64.  Returns the per-step wall times and the process count."""
    import multiprocessing as mp
    cores = host_cores()
    procs = max(1, min(cores, int(host_mem_available_gb() // 3.2), 64))
    ctx = mp.get_context("spawn")
    old = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "1"
    try:
        barrier = ctx.Barrier(procs)
        results = ctx.Queue()
        ps = [ctx.Process(target=_oracle_worker, args=(barrier, results, nsteps)) for _ in range(procs)]
        for p in ps:
            p.start()
        spans = [results.get(timeout=timeout_s) for _ in range(procs * nsteps)]
        for p in ps:
            p.join(timeout=60)
    finally:
        if old is None:
            os.environ.pop("OMP_NUM_THREADS", None)
        else:
            os.environ["OMP_NUM_THREADS"] = old
    walls = []
    for i in range(nsteps):
        st = [(t0, t1) for j, t0, t1 in spans if j == i]
        walls.append(max(t1 for _, t1 in st) - min(t0 for t0, _ in st))
    return {"walls": walls, "procs": procs, "host_cores": cores,
            "value": procs * ORACLE_SAMPLE_FRAMES * LBLOCK / statistics.median(walls) / 1e9}


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on the host cores (one
    single-threaded process per core, each on its own 2^25-sample sample of the
    workload per step); rank 0 only."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    nwarm = 1 if args.warmup >= 1 else 0
    ac = cpu_baseline_allcores(nsteps=nwarm + args.steps)
    walls = ac["walls"][nwarm:]
    total = sum(walls)
    per_step = ac["procs"] * ORACLE_SAMPLE_FRAMES * LBLOCK
    value = args.steps * per_step / total / 1e9
    sample = (f"{ac['procs']} single-threaded processes of {ac['host_cores']} host cores, each "
              f"{ORACLE_SAMPLE_FRAMES} spectra x lblock {LBLOCK} of the workload per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD + f" (sample: {sample})"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ac["procs"], "kind": "oracle", "sample": sample,
                         "nproc": ac["host_cores"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- our arm
def make_inputs(torch, ipfb, dev):
    from paper_2608_23441_b300 import synth
    x = synth.stream_config(LBLOCK, NFRAMES, 2, ntones=16).astype(np.float32)
    xg = torch.from_numpy(x).to(dev)
    del x
    w = torch.from_numpy(ipfb.sinc_hamming_window(LBLOCK, NTAP)).to(dev)
    codes, scale, spec = ipfb.pfb_forward(xg, w, return_spectra=True)
    # phi^2 = quantization noise variance / spectrum variance, from the simulation
    # (setup only, outside the timed path)
    s = scale.double()
    sub = slice(0, 4096)
    q = codes[sub]
    lo = (q & 0xF).to(torch.int16)
    hi = (q >> 4).to(torch.int16)
    lo = torch.where(lo >= 8, lo - 16, lo).double()
    hi = torch.where(hi >= 8, hi - 16, hi).double()
    sp = spec[sub, : LBLOCK // 2]
    err = (lo * s[: LBLOCK // 2] - sp.real.double()) ** 2 + (hi * s[: LBLOCK // 2] - sp.imag.double()) ** 2
    err[:, 0] = (lo[:, 0] * s[0] - sp[:, 0].real.double()) ** 2
    pw = sp.real.double() ** 2 + sp.imag.double() ** 2
    phi2 = float(err.sum() / pw.sum())
    del spec
    return xg, w, codes, scale, phi2


def cufft_pipeline(torch, codes, scale, w, phi2, upfactor):
    """The benchmark step written with torch.fft (cuFFT) and torch's elementwise
    kernels, timed only as a comparison: unpack the 4-bit codes times the channel
    steps, N-point inverse real FFT per spectrum, per phase column a real FFT along
    frames, the Wiener gain G = W (1 + phi^2) / (|W|^2 + phi^2) with W the sub-filter
    eigenvalues of Sec. 3.1 (Eq. decorrelation with Eq. wiener weights; G is
    Hermitian in k, so half the modes suffice), the inverse real FFT, then the real
    FFT of every upfactor * N-sample block.  G is formed once, outside the returned
    step.  Returns step() -> spectra [nblocks, upfactor N / 2 + 1] complex64."""
    J, half = codes.shape
    N = 2 * half
    dev = codes.device
    k = torch.arange(J // 2 + 1, dtype=torch.float64, device=dev)
    W = torch.zeros((J // 2 + 1, N), dtype=torch.complex128, device=dev)
    for r in range(w.shape[0]):
        ang = -2.0 * math.pi * torch.remainder(r * k, J) / J
        W += torch.polar(torch.ones_like(ang), ang)[:, None] * w[r].double()[None, :]
    G = (W * (1.0 + phi2) / (W.abs() ** 2 + phi2)).to(torch.complex64)
    del W
    s = scale.float()
    L = upfactor * N
    nb = (J * N) // L

    def step():
        lo = (codes & 0xF).to(torch.int16)
        hi = (codes >> 4).to(torch.int16)
        lo = torch.where(lo >= 8, lo - 16, lo).float()
        hi = torch.where(hi >= 8, hi - 16, hi).float()
        re = torch.zeros((J, half + 1), dtype=torch.float32, device=dev)
        im = torch.zeros_like(re)
        re[:, :half] = lo
        re[:, half] = hi[:, 0]
        im[:, 1:half] = hi[:, 1:]
        d = torch.fft.irfft(torch.complex(re * s, im * s), n=N, dim=1)
        x = torch.fft.irfft(torch.fft.rfft(d, dim=0) * G, n=J, dim=0)
        return torch.fft.rfft(x.reshape(-1)[: nb * L].reshape(nb, L), dim=1)

    return step


def run_cufft_comparison(torch, codes, scale, w, phi2, ours, reps=5):
    """Time cufft_pipeline on the benchmark's resident codes (CUDA events, after two
    warm-up runs) and compare its spectra with the library's."""
    stream = torch.cuda.current_stream()
    step = cufft_pipeline(torch, codes, scale, w, phi2, UPFACTOR)
    for _ in range(2):
        spec = step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        spec = step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    rel = float(torch.linalg.norm(spec - ours) / torch.linalg.norm(ours))
    del spec, step
    try:
        torch.backends.cuda.cufft_plan_cache.clear()  # the plans' work areas
    except Exception:
        pass
    torch.cuda.empty_cache()
    return {"what": "the same step with torch.fft (cuFFT) and torch elementwise kernels; the Wiener gain "
                    "precomputed outside the timed steps", "ms": ms, "gsas": NSAMP / (ms * 1e-3) / 1e9,
            "ours_ms": None, "rel_diff_to_ours": rel}


ML_LBLOCK, ML_NFRAMES = 4096, 8192


def ml_inputs(torch, ipfb, dev, seed=4):
    """Config-4 instance: lblock 4096, ntap 4, 8192 spectra, 10 % of samples saved as
    64 chunks at seeded offsets, prior values = the true stream, sigma^2 measured."""
    from paper_2608_23441_b300 import synth
    N, J = ML_LBLOCK, ML_NFRAMES
    x = synth.stream_config(N, J, seed).astype(np.float32)
    xg = torch.from_numpy(x).to(dev)
    w = torch.from_numpy(ipfb.sinc_hamming_window(N, NTAP)).to(dev)
    codes, scale, _ = ipfb.pfb_forward(xg, w)
    starts, L = synth.prior_chunks(N * J, 64, 0.1, seed)
    mask = torch.from_numpy(synth.mask_from_chunks(N * J, starts, L)).to(dev)
    # sigma^2 of the quantization noise in d units: exact inverse of the codes vs the
    # true polyphase data, measured with the library's own kernels (setup only)
    xr = ipfb.ipfb_wiener(codes, scale, w, 0.0)
    # d - C x_true = C (x_r - x_true) for the periodic model; its variance, computed by
    # re-running the forward polyphase sum through pfb_forward's spectra would need
    # extra entry points, so use the equivalent |W|-weighted error: var(C e)
    e = (xr - xg).reshape(J, N).double()
    wd = w.double()
    ce = sum(wd[r][None, :] * torch.roll(e, -r, dims=0) for r in range(NTAP))
    sig2 = float(ce.var())
    return codes, scale, w, mask, xg, sig2


def train_learned(torch, dev, epochs=None, seeds=range(1000, 1008)):
    """Learned-preconditioner training with the library's kernels (config-5 recipe,
    8 seeded instances x 5 plain-CG iterates x 50 column pairs = 2000 pairs)."""
    from paper_2608_23441_b300 import precond_train as pt
    epochs = pt.EPOCHS if epochs is None else epochs
    t0 = time.time()
    xin, tgt, info = pt.make_training_set(torch, dev, list(seeds))
    torch.cuda.synchronize()
    t1 = time.time()
    theta, hist = pt.train(torch, dev, xin, tgt, epochs=epochs)
    torch.cuda.synchronize()
    t2 = time.time()
    info.update({"epochs": epochs, "batch": 16, "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1],
                 "data_s": t1 - t0, "train_s": t2 - t1, "loss": "mean (g - (e - u)/s)^2",
                 "seeds": f"{min(seeds)}-{max(seeds)}"})
    del xin, tgt
    return theta, info


NET_FROM_SWEEP = (2, 8, 14, 20)


def run_ml(torch, ipfb, dev, reps=3, theta=None):
    """Time to relative residual 1e-6 per column on the config-4 instance (seed 4, held
    out from training): plain CG, Wiener-PCG and, with theta, the learned FCG."""
    codes, scale, w, mask, prior, sig2 = ml_inputs(torch, ipfb, dev)
    out = {"workload": "ML CG lblock=4096 ntap=4 nframes=8192, 10% prior in 64 chunks, tol 1e-6 per column",
           "noise_var": sig2}
    stream = torch.cuda.current_stream()
    g = ipfb.geom(ML_LBLOCK, NTAP, ML_NFRAMES)
    from paper_2608_23441_b300 import precond_train as pt
    zero = torch.from_numpy(pt.init_theta(0, scale3=0.0)).to(dev)
    names = ("none", "wiener") + (("learned", "learned_g0") if theta is not None else ())
    for name in names:
        learned = name.startswith("learned")
        op = ipfb.OP_ML_LEARNED if learned else ipfb.OP_ML
        ws = torch.empty(ipfb.workspace_size(g, op), dtype=torch.uint8, device=dev)
        kw = dict(precond="learned" if learned else name, tol=1e-6, max_iter=4000, workspace=ws,
                  net=(theta if name == "learned" else zero) if learned else None,
                  net_from=pt.NET_FROM if learned else 0)
        ipfb.ml_solve(codes, scale, w, sig2, mask, prior, **kw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            x, it, res = ipfb.ml_solve(codes, scale, w, sig2, mask, prior, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(x - prior) / torch.linalg.norm(prior))
        out[name] = {"ms": e0.elapsed_time(e1) / reps, "iters_max": int(it.max()), "iters_mean": float(it.float().mean()),
                     "resid_true_max": float(res[1].max()), "rel_error_vs_truth": err}
        del ws
    if theta is not None:
        out["learned_vs_plain_time"] = out["learned"]["ms"] / out["none"]["ms"]
        out["learned_net_from"] = pt.NET_FROM
        out["learned_g0_note"] = "the same learned solve with a zero-output net (g = 0: the Wiener term alone)"
        # the trade-off in net_from: the net's iterations cost far more than the on-chip
        # Wiener-only ones, so joining early saves iterations and joining late saves time
        sweep = []
        ws = torch.empty(ipfb.workspace_size(g, ipfb.OP_ML_LEARNED), dtype=torch.uint8, device=dev)
        for nf in NET_FROM_SWEEP:
            row = {"net_from": nf}
            for key, net in (("learned", theta), ("g0", zero)):
                kw = dict(precond="learned", tol=1e-6, max_iter=4000, workspace=ws, net=net, net_from=nf)
                ipfb.ml_solve(codes, scale, w, sig2, mask, prior, **kw)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    x, it, res = ipfb.ml_solve(codes, scale, w, sig2, mask, prior, **kw)
                e1.record(stream)
                torch.cuda.synchronize()
                row[key] = {"ms": e0.elapsed_time(e1) / reps, "iters_max": int(it.max()),
                            "iters_mean": float(it.float().mean()), "resid_true_max": float(res[1].max())}
            sweep.append(row)
        del ws
        out["learned_net_from_sweep"] = sweep
    out["paper_protocol"] = run_ml_paper_protocol(torch, ipfb, dev, codes, scale, w, prior, sig2, reps=reps)
    del codes, scale, w, mask, prior
    out["paper_size"] = run_ml_long(torch, ipfb, dev, reps=reps)
    return out


def run_ml_long(torch, ipfb, dev, reps=3, seed=11, N=2048, J=65536):
    """The paper's size (Sec. 4.3: 2048-point 4-tap PFB over 65536 frames, 2^27 samples):
    one ML solve of the whole run's circulant system to 1e-6 per column (past the
    on-chip column run the CG vectors stay in HBM), plain CG and Wiener-PCG; 10 % of the
    samples saved as 256 chunks, prior values = the true stream, sigma^2 measured as in
    ml_inputs.  The overlap-save solve (chunks of 8192 frames, 512-frame margins) of the
    same instance is timed beside it."""
    from paper_2608_23441_b300 import synth
    x = synth.gaussian_stream_torch(N * J, seed, dev)
    w = torch.from_numpy(ipfb.sinc_hamming_window(N, NTAP)).to(dev)
    codes, scale, _ = ipfb.pfb_forward(x, w)
    xr = ipfb.ipfb_wiener(codes, scale, w, 0.0)
    e = (xr - x).reshape(J, N).double()
    wd = w.double()
    sig2 = float(sum(wd[r][None, :] * torch.roll(e, -r, dims=0) for r in range(NTAP)).var())
    del e, xr
    starts, L = synth.prior_chunks(N * J, 256, 0.1, seed)
    mask = torch.from_numpy(synth.mask_from_chunks(N * J, starts, L)).to(dev)
    out = {"workload": f"ML CG lblock={N} ntap={NTAP} nframes={J} (2^27 samples), 10% prior in 256 chunks, "
                       "tol 1e-6 per column", "noise_var": sig2}
    stream = torch.cuda.current_stream()
    ws = torch.empty(ipfb.workspace_size(ipfb.geom(N, NTAP, J), ipfb.OP_ML), dtype=torch.uint8, device=dev)
    xn = float(torch.linalg.norm(x))

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, r

    for pre in ("wiener", "none"):
        ms, (xm, it, res) = timed(lambda: ipfb.ml_solve(codes, scale, w, sig2, mask, x, precond=pre, tol=1e-6,
                                                        max_iter=4000, workspace=ws))
        out[pre] = {"ms": ms, "gsas": N * J / (ms * 1e-3) / 1e9, "iters_max": int(it.max()),
                    "iters_mean": float(it.float().mean()), "resid_max": float(res[0].max()),
                    "resid_true_max": float(res[1].max()),
                    "rel_error_vs_truth": float(torch.linalg.norm(xm - x)) / xn}
    del ws
    chunk, margin = 8192, 512
    wss = torch.empty(ipfb.workspace_size(ipfb.geom(N, NTAP, chunk), ipfb.OP_ML_STREAM), dtype=torch.uint8,
                      device=dev)
    ms, (xs, its, rs) = timed(lambda: ipfb.ml_solve_stream(codes, scale, w, sig2, mask, x, chunk, margin,
                                                           precond="wiener", tol=1e-6, max_iter=4000, workspace=wss))
    ref = x[margin * N:(J - margin) * N]
    out["overlap_save_wiener"] = {"chunk": chunk, "margin": margin, "ms": ms, "iters_max": int(its.max()),
                                  "rel_error_vs_truth": float(torch.linalg.norm(xs - ref) / torch.linalg.norm(ref)),
                                  "note": "solves each 8192-frame chunk as a periodic system; "
                                          "the run's first and last 512 frames are not produced"}
    del wss, x, codes, mask
    return out


def run_stream(torch, ipfb, dev, codes, scale, w, phi2, chunk=8192, margin=128, reps=3):
    """Overlap-save Wiener inverse of the 65536-spectrum run in chunks of 8192 with a
    128-frame margin (ipfb_wiener_stream), against the one-block inverse of the run."""
    N = LBLOCK
    out = torch.empty((NFRAMES - 2 * margin) * N, dtype=torch.float32, device=dev)
    g = ipfb.geom(N, NTAP, chunk)
    ws = torch.empty(ipfb.workspace_size(g, ipfb.OP_WIENER_STREAM), dtype=torch.uint8, device=dev)
    ipfb.ipfb_wiener_stream(codes, scale, w, phi2, chunk, margin, out=out, workspace=ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        ipfb.ipfb_wiener_stream(codes, scale, w, phi2, chunk, margin, out=out, workspace=ws)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    full = ipfb.ipfb_wiener(codes, scale, w, phi2)
    ref = full[margin * N:(NFRAMES - margin) * N]
    rel = float(torch.linalg.norm(out - ref) / torch.linalg.norm(ref))
    del ws, full
    return {"chunk": chunk, "margin": margin, "ms": ms, "gsas": out.numel() / (ms * 1e-3) / 1e9,
            "rel_diff_to_one_block_inverse": rel}


def run_ml_paper_protocol(torch, ipfb, dev, codes, scale, w, truth, sig2, reps=3, phi2=0.0141):
    """Sec. 4.3 sample-saving protocol on the config-4 instance: every 4th sample of the
    L central sub-filter paths saved (beta = L / (4 N) = 1 %, 3 %, 10 %), the Wiener
    inverse as the initial guess, then 25 plain-CG iterations of Eq. chi squared with
    unit weights on both terms; timed as one step (ipfb_wiener + ml_solve)."""
    from paper_2608_23441_b300 import synth
    N, J = ML_LBLOCK, ML_NFRAMES
    g = ipfb.geom(N, NTAP, J)
    ws = torch.empty(ipfb.workspace_size(g, ipfb.OP_ML), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    res = {"recipe": "every 4th frame of the L central sub-filter paths, Wiener start (phi^2 0.0141), "
                     "25 plain-CG iterations, unit weights on the data and prior terms (prior weight 1/sigma^2)"}
    tn = float(torch.linalg.norm(truth))
    for beta in (0.01, 0.03, 0.10):
        L = synth.saved_paths(N, beta)
        mask = torch.from_numpy(synth.path_sample_mask(N, J, L)).to(dev)

        def step():
            x0 = ipfb.ipfb_wiener(codes, scale, w, phi2)
            x, _, _ = ipfb.ml_solve(codes, scale, w, sig2, mask, truth, prior_weight=1.0 / sig2, tol=0.0,
                                    max_iter=25, x0=x0, workspace=ws)
            return x0, x
        step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            x0, x = step()
        e1.record(stream)
        torch.cuda.synchronize()
        res[f"beta_{beta:.2f}"] = {"paths": L, "ms": e0.elapsed_time(e1) / reps,
                                   "rel_error_wiener_start": float(torch.linalg.norm(x0 - truth)) / tn,
                                   "rel_error_after_25": float(torch.linalg.norm(x - truth)) / tn}
    del ws
    return res


def run_batched(torch, ipfb, dev, reps=5, seed=3, nstreams=256):
    """Batched-uneven-streams configuration: 256 streams, lblock U{1024, 2048, 4096},
    nframes round(logU[1024, 16384]), ntap 4, 4-bit codes of Gaussian noise from the
    library's forward PFB; inverted by one graph-captured batched run."""
    import tempfile
    from paper_2608_23441_b300 import synth
    geoms = synth.batched_geometries(nstreams, seed)
    streams = []
    total = 0
    for i, (N, J) in enumerate(geoms):
        x = synth.gaussian_stream_torch(N * J, seed * 100003 + i, dev)
        w = torch.from_numpy(ipfb.sinc_hamming_window(N, NTAP)).to(dev)
        codes, scale, _ = ipfb.pfb_forward(x, w)
        del x
        streams.append({"codes": codes, "scale": scale, "window": w, "noise_level": 0.0141})
        total += N * J
    plan = ipfb.BatchedPlan(streams)
    plan.prepare()
    cache = os.path.join(tempfile.gettempdir(), "ipfb_batched_tune.txt")
    t0 = time.perf_counter()
    plan.autotune(cache)
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.run()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            plan.run()
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    out = {"workload": f"{nstreams} streams, lblock U{{1024,2048,4096}}, nframes logU[1024,16384], ntap 4 "
                       f"(seed {seed}), {total} samples", "samples": total, "ms": ms,
           "gsas": total / (ms * 1e-3) / 1e9, "autotune_s": tune_s,
           "variants": {str(2048 << c): plan.variant(2048 << c) for c in range(5)},
           "graph": "one CUDA graph replay per batch (counter reset + 4 persistent kernels)"}
    plan.close()
    return out


def run_ours(args):
    import torch
    from paper_2608_23441_b300 import ipfb
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init(ws)

    xg, w, codes, scale, phi2 = make_inputs(torch, ipfb, dev)
    g = ipfb.geom(LBLOCK, NTAP, NFRAMES)
    wsp = torch.empty(ipfb.workspace_size(g, ipfb.OP_WIENER_UPCHAN), dtype=torch.uint8, device=dev)
    L = UPFACTOR * LBLOCK
    nb = NFRAMES // UPFACTOR
    out = torch.empty((nb, L // 2 + 1), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        ipfb.ipfb_wiener_upchannelize(codes, scale, w, phi2, UPFACTOR, out=out, workspace=wsp)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    # ---- device-timed region (inputs resident; every buffer > L2, so no flush needed)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ipfb.stage_timing(True)
    props = torch.cuda.get_device_properties(dev)
    pci = f"{props.pci_domain_id:08x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0"
    with ClockSampler(local, pci) as clk:
        barrier(dist, torch)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()   # the sampler runs until the timed work has finished
        barrier(dist, torch)
    ms = e0.elapsed_time(e1) / args.steps
    stages = ipfb.stage_times()
    ipfb.stage_timing(False)
    ms_max = max_over_ranks(dist, torch, ms)
    launches = sum(c for _, c in stages.values())

    # ---- end to end through host buffers (pinned), copies inside the timed region.
    # A streaming pipeline over steps: step i's codes go up on one stream, its
    # inverse + up-channelization runs on a second, its spectra come back on a third,
    # so step i's read-back overlaps step i+1's upload and compute.  Two device slots
    # for codes and spectra; every step copies its own inputs in and its own result out.
    h_codes = torch.empty(codes.shape, dtype=codes.dtype, pin_memory=True)
    h_codes.copy_(codes)
    h_out = torch.empty(out.shape, dtype=out.dtype, pin_memory=True)
    d_codes = [torch.empty_like(codes) for _ in range(2)]
    d_out = [out, torch.empty_like(out)]
    s_up, s_cmp, s_down = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev_up = [torch.cuda.Event() for _ in range(2)]
    ev_cmp = [torch.cuda.Event() for _ in range(2)]
    ev_down = [torch.cuda.Event() for _ in range(2)]

    def e2e_steps(n):
        for i in range(n):
            k = i % 2
            with torch.cuda.stream(s_up):
                if i >= 2:
                    s_up.wait_event(ev_cmp[k])          # slot k's codes consumed
                d_codes[k].copy_(h_codes, non_blocking=True)
                ev_up[k].record(s_up)
            with torch.cuda.stream(s_cmp):
                s_cmp.wait_event(ev_up[k])
                if i >= 2:
                    s_cmp.wait_event(ev_down[k])        # slot k's spectra read back
                ipfb.ipfb_wiener_upchannelize(d_codes[k], scale, w, phi2, UPFACTOR, out=d_out[k], workspace=wsp)
                ev_cmp[k].record(s_cmp)
            with torch.cuda.stream(s_down):
                s_down.wait_event(ev_cmp[k])
                h_out.copy_(d_out[k], non_blocking=True)
                ev_down[k].record(s_down)

    torch.cuda.synchronize()
    e2e_steps(2)
    torch.cuda.synchronize()
    barrier(dist, torch)
    e0.record(s_up)
    e2e_steps(args.steps)
    s_down.wait_stream(s_up)
    s_down.wait_stream(s_cmp)
    e1.record(s_down)
    torch.cuda.synchronize()
    barrier(dist, torch)
    ms_e2e = max_over_ranks(dist, torch, e0.elapsed_time(e1) / args.steps)
    del d_out[1]

    # ---- forward PFB (the simulation step), reported as a stage
    fcodes = torch.empty_like(codes)
    ipfb.stage_timing(True)
    for _ in range(3):
        ipfb.pfb_forward(xg, w)
    torch.cuda.synchronize()
    ipfb.stage_timing(True)
    e0.record(stream)
    nf = max(3, args.steps // 2)
    for _ in range(nf):
        ipfb.pfb_forward(xg, w)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_fwd = e0.elapsed_time(e1) / nf
    fstages = ipfb.stage_times()
    ipfb.stage_timing(False)
    del fcodes

    # ---- roofline of the dominant kernel
    peak, peak_kind = measured_peaks()
    T = NSAMP
    alg_bytes = {
        "k2_unpack_irfft": T * 0.5 + T * 4.0,
        "k3_column_wiener": T * 8.0,
        "k4_upchan": T * 4.0 + nb * (L // 2 + 1) * 8.0,
        # the two-pass up-channelizer: each pass reads and writes the whole block set
        # once (scratch in, scratch out in place; scratch in, spectra out)
        "k4a_upchan_frames": T * 8.0,
        "k4b_upchan_pairs": T * 4.0 + nb * (L // 2 + 1) * 8.0,
    }
    per_kernel = {}
    for k, (tot, cnt) in stages.items():
        avg = tot / max(1, cnt)
        ab = alg_bytes.get(k)
        per_kernel[k] = {"avg_ms": avg, "launches": cnt, "share": tot / sum(t for t, _ in stages.values()),
                         "alg_bytes": ab, "achieved_gbs": (ab / (avg * 1e-3) / 1e9) if ab else None}
    dom = max(stages.items(), key=lambda kv: kv[1][0])[0]
    dk = per_kernel[dom]
    traffic = ncu_traffic(dom)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": dk["achieved_gbs"], "peak": peak, "unit": "GB/s",
                "frac": dk["achieved_gbs"] / peak, "traffic": traffic, "peak_source": peak_kind,
                "alg_bytes_per_launch": dk["alg_bytes"], "avg_launch_ms": dk["avg_ms"]}

    value = aggregate_gsas(ws, ms_max)
    e2e_value = aggregate_gsas(ws, ms_e2e)
    pipe_bytes = T * 0.5 + nb * (L // 2 + 1) * 8.0
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (Gaussian + 16 tones, seed 2, 4-bit quantized)",
        "config": {"workload": WORKLOAD, "lblock": LBLOCK, "ntap": NTAP, "nframes": NFRAMES,
                   "upfactor": UPFACTOR, "noise_level": phi2, "parallelism": f"replicas x{ws}",
                   "l2": "inputs and outputs larger than L2 (128 MiB codes, 1 GiB scratch, 1.07 GB spectra)"},
        "roofline": roofline,
        "pipeline_alg_fraction": {"bytes_per_step": pipe_bytes,
                                  "frac": pipe_bytes / (ms * 1e-3) / 1e9 / peak},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(codes.numel()),
                "d2h_bytes_per_step": int(out.numel() * 8), "ms_per_step": ms_e2e,
                "pipeline": "pinned host codes -> device, ipfb_wiener_upchannelize, spectra -> pinned host; "
                            "three streams, two device slots, step i's read-back overlapping step i+1"},
        "gpu_launches": int(launches),
        "kernels": per_kernel,
        "stages": {"pfb_forward_ms": ms_fwd, "pfb_forward_gsas": NSAMP / (ms_fwd * 1e-3) / 1e9,
                   "pfb_forward_kernels": {k: {"avg_ms": t / max(1, c), "launches": c}
                                           for k, (t, c) in fstages.items()}},
        "clocks": clk.summary(),
    }
    result["stages"]["stream_overlap_save"] = run_stream(torch, ipfb, dev, codes, scale, w, phi2)
    if not args.no_cufft:
        try:
            cmp = run_cufft_comparison(torch, codes, scale, w, phi2, out)
            cmp["ours_ms"] = ms
            result["cufft_comparison"] = cmp
        except Exception as exc:  # a comparison only: its failure must not cost the benchmark line
            result["cufft_comparison"] = {"error": repr(exc)[:300]}
            torch.cuda.empty_cache()
    if not args.no_ml:
        theta, tinfo = (None, None) if args.no_learned else train_learned(torch, dev)
        result["ml"] = run_ml(torch, ipfb, dev, theta=theta)
        if tinfo is not None:
            result["ml"]["training"] = tinfo
    if not args.no_batched:
        del xg
        torch.cuda.empty_cache()
        result["batched"] = run_batched(torch, ipfb, dev)
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline_measure(1)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_profile_case(lblock: int, nframes: int, reps: int):
    """A smaller case of the same pipeline for ncu captures: `reps` forward PFBs of
    a Gaussian stream, then `reps` calls of ipfb_wiener_upchannelize (upfactor 64)."""
    import torch
    from paper_2608_23441_b300 import ipfb, synth
    dev = torch.device("cuda", 0)
    x = torch.from_numpy(synth.gaussian_stream(lblock * nframes, 1).astype(np.float32)).to(dev)
    w = torch.from_numpy(ipfb.sinc_hamming_window(lblock, NTAP)).to(dev)
    for _ in range(reps):
        codes, scale, _ = ipfb.pfb_forward(x, w)
    for _ in range(reps):
        ipfb.ipfb_wiener_upchannelize(codes, scale, w, 0.014, UPFACTOR)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": {"lblock": lblock, "nframes": nframes, "reps": reps}}))
    return 0


def run_profile_ml_long(lblock: int, nframes: int, reps: int):
    """A smaller case of the long-column ML solve for ncu (whole-graph captures): the
    run_ml_long instance at lblock x nframes, `reps` Wiener-PCG solves to 1e-6."""
    import torch
    from paper_2608_23441_b300 import ipfb, synth
    dev = torch.device("cuda", 0)
    N, J = lblock, nframes
    x = synth.gaussian_stream_torch(N * J, 11, dev)
    w = torch.from_numpy(ipfb.sinc_hamming_window(N, NTAP)).to(dev)
    codes, scale, _ = ipfb.pfb_forward(x, w)
    starts, L = synth.prior_chunks(N * J, 256, 0.1, 11)
    mask = torch.from_numpy(synth.mask_from_chunks(N * J, starts, L)).to(dev)
    ws = torch.empty(ipfb.workspace_size(ipfb.geom(N, NTAP, J), ipfb.OP_ML), dtype=torch.uint8, device=dev)
    for _ in range(reps):
        xm, it, res = ipfb.ml_solve(codes, scale, w, 0.0114, mask, x, precond="wiener", tol=1e-6, max_iter=4000,
                                    workspace=ws)
    torch.cuda.synchronize()
    print(json.dumps({"profile_ml_long": {"lblock": N, "nframes": J, "reps": reps, "iters_max": int(it.max()),
                                          "iters_sum": int(it.sum())}}))
    return 0


def run_profile_batched(nstreams: int):
    """The batched-streams configuration (first `nstreams` streams of the seeded
    256-stream recipe) planned with the default variants and run once, for ncu
    captures of the batched kernels."""
    import torch
    from paper_2608_23441_b300 import ipfb, synth
    dev = torch.device("cuda", 0)
    geoms = synth.batched_geometries(256, 3)[:nstreams]
    streams = []
    for i, (N, J) in enumerate(geoms):
        x = synth.gaussian_stream_torch(N * J, 3 * 100003 + i, dev)
        w = torch.from_numpy(ipfb.sinc_hamming_window(N, NTAP)).to(dev)
        codes, scale, _ = ipfb.pfb_forward(x, w)
        del x
        streams.append({"codes": codes, "scale": scale, "window": w, "noise_level": 0.0141})
    plan = ipfb.BatchedPlan(streams)
    plan.prepare()
    plan.run()
    torch.cuda.synchronize()
    print(json.dumps({"profile_batched": {"streams": nstreams, "samples": int(sum(N * J for N, J in geoms))}}))
    plan.close()
    return 0


def run_profile_net(nslots: int):
    """One learned-preconditioner net forward over `nslots` columns of 8192 frames
    (the ML workload's column length), seeded inputs and He-initialised weights, for
    ncu captures of the net kernels."""
    import torch
    from paper_2608_23441_b300 import ipfb, precond_train
    dev = torch.device("cuda", 0)
    g = torch.Generator(device="cpu").manual_seed(5)
    xin = torch.randn((nslots, 2, ML_NFRAMES), generator=g).to(dev)
    xin[:, 1] = (xin[:, 1] > 1.0).float()
    theta = torch.from_numpy(precond_train.init_theta(5, scale3=1.0)).to(dev)
    y = ipfb.net_forward(theta, xin)
    torch.cuda.synchronize()
    print(json.dumps({"profile_net": {"slots": nslots, "frames": ML_NFRAMES, "y_rms": float(y.pow(2).mean().sqrt())}}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ml", action="store_true", help="skip the ML (config-4) timing")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip training the learned preconditioner and its ML timing")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-streams timing")
    ap.add_argument("--no-cufft", action="store_true", help="skip the torch.fft (cuFFT) comparison")
    ap.add_argument("--profile-ml-long", nargs=3, type=int, metavar=("LBLOCK", "NFRAMES", "REPS"),
                    help="run only a smaller long-column ML solve (for ncu captures)")
    ap.add_argument("--profile-case", nargs=3, type=int, metavar=("LBLOCK", "NFRAMES", "REPS"),
                    help="run a smaller case of the pipeline (for ncu captures) and exit")
    ap.add_argument("--profile-batched", type=int, metavar="NSTREAMS",
                    help="plan and run the first NSTREAMS streams of the batched configuration once (for ncu)")
    ap.add_argument("--profile-net", type=int, metavar="NSLOTS",
                    help="run one net forward over NSLOTS columns of 8192 frames (for ncu)")
    args = ap.parse_args()
    if args.profile_net:
        return run_profile_net(args.profile_net)
    if args.profile_case:
        return run_profile_case(*args.profile_case)
    if args.profile_ml_long:
        return run_profile_ml_long(*args.profile_ml_long)
    if args.profile_batched:
        return run_profile_batched(args.profile_batched)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
