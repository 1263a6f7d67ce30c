#!/usr/bin/env python3
"""Benchmark of the DPF-PIR server hot path on GB300.

One step = one pass of the whole server path over one batch of queries:
key ingest from device memory, DPF full-domain expansion (AES-128 PRF) fused
with the share x table product mod 2^32, and the reduction into the output
shares (pir_server_eval_device).  The default workload is the largest
single-GPU configuration: a 2^24-row table of 32 u32 words (2 GiB), 1024
queries per step.  After its timed region that run also measures the other
configurations compactly (plain single query, batched 2^20 x 64, the 8-table
mix, the serving loop at two offered rates) under "other_configs".  Inputs are
seeded synthetic data (workloads/).

Prints ONE JSON line (rank 0).  Under torchrun each rank drives its own GPU
with its own queries and table copy (queries are independent: weak scaling,
no data-path collective); the process group only carries the barrier and the
max-over-ranks timing.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   (the CPU oracle on the host cores)
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import re
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "PIR queries/sec per server (bit-exact) and p50/p99 latency; plain vs batched/served"
WORKLOADS = {
    "batched_1m": dict(rows=1 << 20, width=64, batch=256, seed=20,
                       desc="batched: 256 queries per step against one 2^20-row x 64-word u32 table "
                            "(256 MiB, 2048-bit entries), AES-128 PRF, fused expand+contract"),
    "plain_64k": dict(rows=1 << 16, width=16, batch=1, seed=16,
                      desc="plain: one query per launch against a 2^16-row x 16-word u32 table (4 MiB)"),
    "large_16m": dict(rows=1 << 24, width=32, batch=1024, seed=24,
                      desc="large: 1024 queries per step against a 2^24-row x 32-word u32 table (2 GiB)"),
    "serving": dict(seed=55, rows=None, width=None,
                    desc="serving: Poisson arrivals over 4 resident tables (2^18x64, 2^20x32, 2^22x32, 2^24x16 "
                         "words, 1,728 MiB), table uniform per query, continuous cross-table batching"),
    "pbr_1m": dict(rows=1 << 20, width=64, bin_rows=1 << 10, seed=21,
                   desc="partial batch retrieval: the 2^20-row x 64-word table (256 MiB) cut into 1024 bins of "
                        "2^10 rows, one DPF query per bin per step (1024 per step), all bins in one launch"),
    "serving_hotfull": dict(seed=57, rows=None, width=None,
                            desc="hot/full split serving: a 2^22-row x 32-word full table (512 MiB) and its 2^18 most "
                                 "popular rows as a hot table, Poisson requests of 10 Zipf(1.1) rows, each sent as "
                                 "exactly 10 hot + 3 full queries"),
    "multi_table": dict(seed=33, rows=None, width=None,
                        desc="multi-table: 2048 queries Zipf(1.1) over 8 tables (2^16..2^22 rows, 16..128 words, "
                             "1,460 MiB), one graph-captured persistent launch per step"),
}
def workload_config(name: str, prf: int, world: int) -> dict:
    """The `config` object of a workload's JSON line: host-side facts only, the
    same for both arms (the product's plan and server settings are reported
    beside it, under `plan` and `server`)."""
    wk = WORKLOADS[name]
    par = f"{world} replica(s), independent queries"
    if name in ("batched_1m", "plain_64k", "large_16m"):
        rows, width = wk["rows"], wk["width"]
        mib = rows * width * 4 >> 20
        return {"workload": wk["desc"], "rows": rows, "width_words": width, "batch": wk["batch"],
                "n": wl.domain_bits(rows), "prf": PRF_NAMES[prf],
                "l2": f"inputs larger than L2: table {mib} MiB per step, no flush" if rows * width * 4 > L2_BYTES
                else "table fits in L2; no flush (resident-table serving)", "parallelism": par}
    if name == "multi_table":
        shapes = list(zip(wl.MULTI_TABLE_ROWS, wl.MULTI_TABLE_WIDTHS))
        assign = wl.zipf_assignment(wk["seed"], len(shapes), wl.MULTI_TABLE_QUERIES)
        return {"workload": wk["desc"], "tables": [{"rows": r, "width_words": w} for r, w in shapes],
                "queries": wl.MULTI_TABLE_QUERIES,
                "queries_per_table": np.bincount(assign, minlength=len(shapes)).tolist(), "prf": "AES-128",
                "tables_mib": round(sum(r * w * 4 for r, w in shapes) / 2**20, 1),
                "l2": "inputs larger than L2 (1,460 MiB of tables per step), no flush", "parallelism": par}
    if name == "pbr_1m":
        rows, width, bin_rows = wk["rows"], wk["width"], wk["bin_rows"]
        return {"workload": wk["desc"], "rows": rows, "width_words": width, "bin_rows": bin_rows,
                "bins": -(-rows // bin_rows), "n_per_bin": wl.domain_bits(bin_rows), "prf": PRF_NAMES[prf],
                "l2": f"inputs larger than L2: table {rows * width * 4 >> 20} MiB per step, no flush",
                "parallelism": par}
    if name == "serving":
        shapes = wl.SERVING_TABLES
        return {"workload": wk["desc"], "tables": [{"rows": r, "width_words": w} for r, w in shapes],
                "tables_mib": round(sum(r * w * 4 for r, w in shapes) / 2**20, 1), "prf": "AES-128",
                "l2": "inputs larger than L2 (1,728 MiB of tables), no flush", "parallelism": par}
    if name == "serving_hotfull":
        full_rows, width = wl.HOTFULL_FULL
        return {"workload": wk["desc"], "full": {"rows": full_rows, "width_words": width},
                "hot": {"rows": wl.HOTFULL_HOT_ROWS, "width_words": width},
                "wanted_per_request": wl.HOTFULL_WANTED, "q_hot": wl.HOTFULL_Q_HOT, "q_full": wl.HOTFULL_Q_FULL,
                "prf": "AES-128", "l2": "inputs larger than L2 (512 MiB full table), no flush",
                "parallelism": f"{world} replica(s), independent requests"}
    raise KeyError(name)


# Paper Table 4 (Sec. 5): 1M entries x 2048 bit, AES-128, one V100: 1,358 QPS (other hardware; context).
PAPER_QPS = {"batched_1m": 1358.0}
L2_BYTES = 129 * 1000 * 1000


def measured_bf16_tflops():
    """Dense bf16 tensor throughput measured on this machine's GPUs (burst), else
    the recipe's fallback figure; fp16 has the same nominal dense rate."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]), "of measured"
    except (OSError, ValueError, KeyError):
        return 1900.0, "of fallback"


def measured_hbm_gbs():
    """HBM copy bandwidth measured on this machine's GPUs (MEASURED_PEAKS.json),
    else the recipe's fallback figure."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "of measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "of fallback"


LOOKUPS_PER_NODE = 360  # table-lookup AES-128: 40 for the key expansion + 2 x 160 for the two blocks
ORACLE_S_PER_NODE = 1.7e-6  # the oracle's cost per tree node on one Grace core, roughly
CHACHA_ALU_OPS_PER_NODE = 640  # ChaCha20 block: 20 rounds x 4 quarter rounds x (4 XOR + 4 rotate)


# ----------------------------------------------------------------------------- distributed plumbing

def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def dist_init(world: int, backend: str):
    if world > 1:
        import torch.distributed as dist

        if not dist.is_initialized():
            dist.init_process_group(backend=backend)


def barrier(world: int, device=None):
    if world > 1:
        import torch.distributed as dist

        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(base: int, rank: int) -> int:
    """Each rank draws its own queries (weak scaling); rank 0 keeps the base seed."""
    return base + 7919 * rank


# ----------------------------------------------------------------------------- clocks

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    """nvidia-smi sampled every 100 ms while the timed region runs."""

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.15)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.12)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), max=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swpc=parts[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swpc", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["max"] for r in rows),
                "power_w_max": max(r["power"] for r in rows), "reasons": sorted(reasons), "samples": len(rows)}


def gpu_id_for(device) -> str | None:
    import torch

    props = torch.cuda.get_device_properties(device)
    bus = getattr(props, "pci_bus_id", None)
    dom = getattr(props, "pci_domain_id", None)
    dev = getattr(props, "pci_device_id", None)
    if bus is None or dom is None or dev is None:
        return None
    return f"{dom:08X}:{bus:02X}:{dev:02X}.0"


# ----------------------------------------------------------------------------- CPU oracle timing

PRFS = {"aes128": 0, "chacha20": 1}
PRF_NAMES = {0: "AES-128", 1: "ChaCha20"}


def _oracle_jobs(rows: int, seed: int, queries: int, parts: int, prf: int):
    """Oracle keys for `queries` seeded queries, each cut into `parts` row ranges
    (the answer is linear over index ranges, Sec. 3.2.7: the parts' shares add up
    to the query's share, so a range is a fair share of one query's work)."""
    import oracle

    n = wl.domain_bits(rows)
    rnd = wl.key_randomness(seed, n, queries)
    alphas = wl.alphas(seed, rows, queries)
    keys = [oracle.gen(n, int(a), 1, r0, r1, c0, prf)[0] for (r0, r1, c0), a in zip(rnd, alphas)]
    cuts = [rows * i // parts for i in range(parts + 1)]
    return [(k, cuts[i], cuts[i + 1]) for k in keys for i in range(parts)]


def oracle_qps(rows: int, width: int, seed: int, table_np, target_cpu_s: float = 20.0, prf: int = 0):
    """Times the oracle (as it stands) on host threads over about `target_cpu_s`
    of CPU work: whole queries (FullEval + inner product) per thread, or, when
    that is fewer queries than threads, each query cut into row ranges so that
    every thread has work.  Returns (qps, threads, queries, wall)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    oracle.build()
    n = wl.domain_bits(rows)
    threads = os.cpu_count() or 1
    per_query_s = ORACLE_S_PER_NODE * (1 << n)
    queries = max(1, min(int(target_cpu_s / per_query_s + 0.5), 64 * threads))
    parts = 1 if queries >= threads else -(-threads // queries)
    jobs = _oracle_jobs(rows, seed + 1, queries, parts, prf)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda j: oracle.answer(j[0], table_np, j[1], j[2]), jobs))
    wall = time.perf_counter() - t0
    return queries / wall, min(threads, len(jobs)), queries, wall


def oracle_one_core_qps(rows: int, seed: int, table_np, prf: int = 0, max_s: float = 6.0):
    """The oracle on one host thread: queries per second over about max_s of
    work (whole queries, or the first rows/parts of one query when a whole one
    takes longer; returns the fraction of a query timed)."""
    import oracle

    oracle.build()
    n = wl.domain_bits(rows)
    per_query_s = ORACLE_S_PER_NODE * (1 << n)
    queries = max(1, min(8, int(max_s / per_query_s)))
    parts = max(1, 1 << max(0, math.ceil(math.log2(per_query_s / max_s)))) if queries == 1 else 1
    jobs = _oracle_jobs(rows, seed + 2, queries, parts, prf)
    if parts > 1:
        jobs = jobs[:1]
    t0 = time.perf_counter()
    for k, lo, hi in jobs:
        oracle.answer(k, table_np, lo, hi)
    frac = (jobs[0][2] - jobs[0][1]) / rows if parts > 1 else queries
    return frac / (time.perf_counter() - t0), frac


def host_cpu_model() -> str:
    """The host CPU as the OS names it (model name, or the Arm part number)."""
    try:
        info = open("/proc/cpuinfo").read()
    except OSError:
        return "unknown"
    arm_parts = {"0xd4f": "Arm Neoverse-V2", "0xd40": "Arm Neoverse-V1", "0xd49": "Arm Neoverse-N2",
                 "0xd0c": "Arm Neoverse-N1"}
    for key in ("model name", "CPU part"):
        for line in info.splitlines():
            if line.lower().startswith(key.lower()):
                value = line.split(":", 1)[1].strip()
                return arm_parts.get(value.lower(), f"{key}: {value}")
    return "unknown"


# ----------------------------------------------------------------------------- our arm

def kernel_source_digest() -> str:
    """sha256[:16] of the fused kernels' device code: dpf_eval.cu up to the end of
    its device namespace (the host-side planner below it does not change what a
    launch of a given shape does), with comments and blank lines removed, so
    that editing a comment keeps the recorded traffic of the same code."""
    src = open(os.path.join(ROOT, "paper_2301_10904_gb300", "csrc", "dpf_eval.cu"), "rb").read()
    code = src[:src.index(b"}  // namespace dev")].decode()
    code = re.sub(r"/\*.*?\*/", "", code, flags=re.S)
    lines = [re.sub(r"//.*$", "", line).rstrip() for line in code.splitlines()]
    return hashlib.sha256("\n".join(line for line in lines if line).encode()).hexdigest()[:16]


def profiled_traffic(workload: str):
    """DRAM bytes per launch of the fused kernel from the committed ncu summary,
    if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(workload)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("kernel_source_sha256_16") != kernel_source_digest():
        return None
    return rec.get("dram_bytes_per_launch")


def client_gen_rate(pir, n: int, count: int, prf: int):
    """Client Gen throughput on the host (Sec. 3.1: Gen is O(log L), Eval O(L)):
    key pairs per second for `count` keys, on one thread and on all of them."""
    count = max(count, 64)
    alphas = [(i * 2654435761) % (1 << n) for i in range(count)]
    res = {"n": n, "keys": count, "prf": PRF_NAMES[prf]}
    for label, threads in (("one_thread", 1), ("all_threads", os.cpu_count() or 1)):
        pir.pir_keygen_batch(n, alphas[:8], None, prf=prf, seed=b"\x11" * 32, threads=threads)  # warm-up
        t0 = time.perf_counter()
        pir.pir_keygen_batch(n, alphas, None, prf=prf, seed=b"\x11" * 32, threads=threads)
        dt = time.perf_counter() - t0
        res[label] = {"key_pairs_per_s": round(count / dt, 1), "us_per_key_pair": round(1e6 * dt / count, 2),
                      "threads": threads}
    return res


def _pack_keys(keys, offsets, total):
    buf = bytearray(total)
    for k, o in zip(keys, offsets):
        buf[int(o):int(o) + len(k)] = k
    return buf


class SingleTableWorkload:
    """One table, one batch of queries per step (pir_server_eval_device)."""

    def __init__(self, name, wk, pir, torch, device, stream, seed, args):
        self.name, self.pir, self.torch, self.device, self.stream, self.args = name, pir, torch, device, stream, args
        self.rows, self.width, self.batch = wk["rows"], wk["width"], wk["batch"]
        self.desc = wk["desc"]
        self.n = pir.pir_domain_bits(self.rows)
        self.kb = pir.pir_key_bytes(self.n)
        self.seed = seed
        self.table = wl.table_u32_torch(seed, self.rows, self.width, device)
        self.alphas = wl.alphas(seed, self.rows, self.batch)
        self.prf = PRFS[args.prf]
        self.pairs = [pir.pir_keygen_prf(self.n, int(a), 1, self.prf, hashlib.sha256(b"bench%d-%d" % (seed, q)).digest())
                      for q, a in enumerate(self.alphas)]
        self.keys0 = b"".join(p[0] for p in self.pairs)
        self.keys1 = b"".join(p[1] for p in self.pairs)
        self.dkeys = torch.frombuffer(bytearray(self.keys0), dtype=torch.uint8).to(device)
        self.dout = torch.empty((self.batch, self.width), dtype=torch.int32, device=device)
        self.plan = pir.pir_plan_for(self.rows, self.width, self.batch)
        self.queries_per_step = self.batch
        self.nodes_per_step = self.batch * ((1 << self.n) - 1)
        self.kernel = "fused_eval_kernel"
        self.h2d_bytes, self.d2h_bytes = self.batch * self.kb, self.batch * self.width * 4
        self.hkeys = torch.frombuffer(bytearray(self.keys0), dtype=torch.uint8).pin_memory()
        self.hout = torch.empty((self.batch, self.width), dtype=torch.int32).pin_memory()
        self.table_desc = pir.table_of(self.table)  # the C descriptor, built once as a C caller would

    def step(self):
        self.pir.pir_server_eval_device(self.table, self.dkeys, self.batch, self.dout, stream=self.stream)

    def e2e_step(self):
        self.pir.pir_server_eval(self.table_desc, self.hkeys, self.batch, self.hout, stream=self.stream)

    def e2e_matches(self):
        return bool(np.array_equal(self.hout.numpy(), self.dout.cpu().numpy()))

    def selfcheck(self):
        torch, pir = self.torch, self.pir
        d1 = torch.empty_like(self.dout)
        k1 = torch.frombuffer(bytearray(self.keys1), dtype=torch.uint8).to(self.device)
        pir.pir_server_eval_device(self.table, k1, self.batch, d1, stream=self.stream)
        torch.cuda.synchronize(self.device)
        rec = (self.dout.cpu().numpy().view(np.uint32).astype(np.uint64) + d1.cpu().numpy().view(np.uint32))
        want = self.table[torch.from_numpy(self.alphas.astype(np.int64)).to(self.device)].cpu().numpy()
        return bool(np.array_equal((rec & 0xFFFFFFFF).astype(np.uint32), want.view(np.uint32)))

    def plan_info(self):
        return self.plan.as_dict()

    def tc_roofline(self, ms, flops, s_bytes):
        """The tcgen05 contraction against both ceilings: its limb products
        (10 fp16 MMAs per u32 multiply-add) against the dense tensor peak, and
        its algorithmic bytes (share matrix + table, each read once) against
        HBM copy bandwidth."""
        tpeak, tbasis = measured_bf16_tflops()
        hpeak, hbasis = measured_hbm_gbs()
        tf = flops / (ms * 1e-3) / 1e12
        gbs = (s_bytes + self.rows * self.width * 4) / (ms * 1e-3) / 1e9
        return {"tensor": {"achieved": round(tf, 1), "peak": tpeak, "unit": "TFLOP/s", "frac": round(tf / tpeak, 4),
                           "peak_basis": tbasis + " (bf16 burst; fp16 dense is the same nominal rate)"},
                "hbm": {"achieved": round(gbs, 1), "peak": hpeak, "unit": "GB/s", "frac": round(gbs / hpeak, 4),
                        "peak_basis": hbasis},
                # the share matrix here is a fresh aligned tensor (ld = rows), so the
                # tensor-map kernel runs unless the environment selects the other one
                "kernel": ("contract_tc_kernel" if os.environ.get("PIR_TC_TENSOR_MAPS", "1").startswith("0")
                           or self.rows % 4 or self.width % 4 else "contract_tc2_kernel"), "ms": round(ms, 4)}

    def extras(self):
        torch, pir, stream = self.torch, self.pir, self.stream
        out = {}
        if self.batch > 1:  # plain path on the same table: one query per launch
            pk = [torch.frombuffer(bytearray(p[0]), dtype=torch.uint8).to(self.device) for p in self.pairs[:32]]
            po = torch.empty((1, self.width), dtype=torch.int32, device=self.device)
            for k in pk[:3]:
                pir.pir_server_eval_device(self.table, k, 1, po, stream=stream)
            torch.cuda.synchronize(self.device)
            lat = []
            for k in pk:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                pir.pir_server_eval_device(self.table, k, 1, po, stream=stream)
                b.record(stream)
                b.synchronize()
                lat.append(a.elapsed_time(b))
            out["plain"] = {"qps": round(1e3 / statistics.mean(lat), 2),
                            "p50_ms": round(float(np.percentile(lat, 50)), 4),
                            "p99_ms": round(float(np.percentile(lat, 99)), 4), "launches": len(lat)}
        s_bytes = self.batch * self.rows * 4
        free_bytes = torch.cuda.mem_get_info(self.device)[0]
        if self.args.materialised and self.batch > 1 and s_bytes <= 0.6 * free_bytes:
            S = torch.empty((self.batch, self.rows), dtype=torch.int32, device=self.device)
            m_imad, m_mma = torch.empty_like(self.dout), torch.empty_like(self.dout)

            def timed(fn, reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                fn()  # warm-up
                a.record(stream)
                for _ in range(reps):
                    fn()
                b.record(stream)
                b.synchronize()
                return a.elapsed_time(b) / reps

            reps = 3 if s_bytes <= (8 << 30) else 1
            exp = timed(lambda: pir.pir_expand_materialise(self.rows, self.dkeys, self.batch, S, stream=stream), reps)
            con = timed(lambda: pir.pir_contract_u32(S, self.batch, self.table, m_imad, stream=stream), reps)
            mma = timed(lambda: pir.pir_contract_u32(S, self.batch, self.table, m_mma,
                                                     engine=pir.PIR_CONTRACT_MMA_U8, stream=stream), reps)
            m_tc = torch.empty_like(self.dout)
            tc = timed(lambda: pir.pir_contract_u32(S, self.batch, self.table, m_tc,
                                                    engine=pir.PIR_CONTRACT_TC_F16, stream=stream), reps)
            ok_imad, ok_mma = bool(torch.equal(m_imad, self.dout)), bool(torch.equal(m_mma, self.dout))
            ok_tc = bool(torch.equal(m_tc, self.dout))
            tot = exp + min(con, mma, tc)
            # 10 fp16 limb products per u32 multiply-add on the tensor pipe: 2 * 10 * B * L * W flops
            tc_flops = 2.0 * 10 * self.batch * self.rows * self.width
            out["materialised"] = {"qps": round(self.batch / (tot / 1e3), 2),
                                   "expand_ms": round(exp, 4),
                                   "contract_imad_ms": round(con, 4),
                                   "contract_mma_u8_ms": round(mma, 4),
                                   "contract_tc_f16_ms": round(tc, 4),
                                   "contract_tc_f16_roofline": self.tc_roofline(tc, tc_flops, s_bytes),
                                   "share_matrix_bytes": s_bytes,
                                   "bit_exact_vs_fused": {"imad": ok_imad, "mma_u8": ok_mma, "tc_f16": ok_tc}}
            del S
        if self.args.scan and self.width % 4 == 0 and self.rows * self.width * 4 > 2 * L2_BYTES:
            out["scan"] = self.scan_roofline()
        out["client_gen"] = client_gen_rate(self.pir, self.n, self.batch, self.prf)
        return out

    def scan_roofline(self):
        """The streaming scan engine (PIR_CONTRACT_SCAN) on the materialised shares
        of 1 and 8 queries: HBM bytes (table + shares + out) per launch / launch time."""
        torch, pir, stream = self.torch, self.pir, self.stream
        peak, basis = measured_hbm_gbs()
        res = {}
        for q in (1, 8):
            if q > self.batch:
                continue
            S = torch.empty((q, self.rows), dtype=torch.int32, device=self.device)
            pir.pir_expand_materialise(self.rows, self.dkeys[:q * self.kb], q, S, stream=stream)
            a = torch.empty((q, self.width), dtype=torch.int32, device=self.device)
            b = torch.empty_like(a)
            pir.pir_contract_u32(S, q, self.table, b, engine=pir.PIR_CONTRACT_IMAD, stream=stream)
            for _ in range(3):
                pir.pir_contract_u32(S, q, self.table, a, engine=pir.PIR_CONTRACT_SCAN, stream=stream)
            reps = 20
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
            for i in range(reps):
                ev[2 * i].record(stream)
                pir.pir_contract_u32(S, q, self.table, a, engine=pir.PIR_CONTRACT_SCAN, stream=stream)
                ev[2 * i + 1].record(stream)
            ev[-1].synchronize()
            ms = statistics.median(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(reps))
            nbytes = self.rows * self.width * 4 + q * self.rows * 4 + q * self.width * 4
            gbs = nbytes / (ms / 1e3) / 1e9
            res[f"q{q}"] = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                            "frac": round(gbs / peak, 4), "ms": round(ms, 4), "bytes_per_launch": nbytes,
                            "kernel": "contract_scan_kernel", "bit_exact_vs_imad": bool(torch.equal(a, b)),
                            "faults": pir.pir_device_status(), "peak_basis": basis}
            del S
        return res

    def cpu_baseline(self):
        table_np = self.table.cpu().numpy().view(np.uint32)
        qps, cores, nq, wall = oracle_qps(self.rows, self.width, self.seed, table_np, prf=self.prf)
        one, n1 = oracle_one_core_qps(self.rows, self.seed, table_np, prf=self.prf)
        split = "" if nq >= cores else f", each cut into {-(-cores // nq)} row ranges over the threads"
        return {"value": round(qps, 4), "unit": "queries/s", "cores": cores, "kind": "oracle",
                "sample": f"{nq} queries of this workload (oracle FullEval + inner product){split}, "
                          f"{cores} host threads, {wall:.1f} s wall",
                "one_core": {"value": round(one, 4),
                             "sample": f"{n1:g} queries on one thread" if n1 >= 1 else
                             f"the first {n1:g} of one query's rows on one thread, scaled to whole queries"},
                "nproc": os.cpu_count(), "cpu": host_cpu_model()}


class MultiTableWorkload:
    """Eight tables of uneven sizes and widths, 2048 queries Zipf(1.1) over them,
    one graph-captured persistent launch per step; item size from the autotuner."""

    def __init__(self, name, wk, pir, torch, device, stream, seed, args):
        self.name, self.pir, self.torch, self.device, self.stream, self.args = name, pir, torch, device, stream, args
        self.desc = wk["desc"]
        self.shapes = list(zip(wl.MULTI_TABLE_ROWS, wl.MULTI_TABLE_WIDTHS))
        self.batch = wl.MULTI_TABLE_QUERIES
        self.seed = seed
        self.assign = wl.zipf_assignment(seed, len(self.shapes), self.batch)
        self.tables = [wl.table_u32_torch(seed * 100 + i, r, w, device) for i, (r, w) in enumerate(self.shapes)]
        rng = np.random.Generator(np.random.PCG64(seed))
        self.alphas = [int(rng.integers(0, self.shapes[t][0])) for t in self.assign]
        self.ns = [pir.pir_domain_bits(r) for r, _ in self.shapes]
        self.pairs = [pir.pir_keygen(self.ns[t], a, 1, hashlib.sha256(b"multi%d-%d" % (seed, q)).digest())
                      for q, (t, a) in enumerate(zip(self.assign, self.alphas))]
        probe = pir.pir_multi_plan_create(self.tables, self.assign)
        self.keys0 = _pack_keys([p[0] for p in self.pairs], probe.key_offsets, probe.key_bytes_total)
        self.keys1 = _pack_keys([p[1] for p in self.pairs], probe.key_offsets, probe.key_bytes_total)
        self.dkeys = torch.frombuffer(bytearray(self.keys0), dtype=torch.uint8).to(device)
        self.dout = torch.empty((probe.out_words_total,), dtype=torch.int32, device=device)
        self.item_log2, self.tune_ms = pir.pir_multi_autotune(self.tables, self.assign, self.dkeys, self.dout,
                                                              stream=stream)
        probe.close()
        self.plan = pir.pir_multi_plan_create(self.tables, self.assign, self.item_log2)
        self.graph = pir.pir_multi_graph_create(self.plan, self.dkeys, self.dout)
        self.queries_per_step = self.batch
        self.nodes_per_step = sum((1 << self.ns[t]) - 1 for t in self.assign)
        self.kernel = "multi_eval_kernel"
        self.h2d_bytes, self.d2h_bytes = self.plan.key_bytes_total, self.plan.out_words_total * 4
        self.hkeys = torch.frombuffer(bytearray(self.keys0), dtype=torch.uint8).pin_memory()
        self.hout = torch.empty((self.plan.out_words_total,), dtype=torch.int32).pin_memory()

    def step(self):
        self.graph.launch(self.stream)

    def e2e_step(self):
        self.pir.pir_server_eval_multi_host(self.plan, self.hkeys, self.hout, stream=self.stream)

    def e2e_matches(self):
        return bool(np.array_equal(self.hout.numpy(), self.dout.cpu().numpy()))

    def selfcheck(self):
        torch, pir = self.torch, self.pir
        d1 = torch.empty_like(self.dout)
        k1 = torch.frombuffer(bytearray(self.keys1), dtype=torch.uint8).to(self.device)
        pir.pir_server_eval_multi(self.plan, k1, d1, stream=self.stream)
        torch.cuda.synchronize(self.device)
        a, b = self.dout.cpu().numpy().view(np.uint32), d1.cpu().numpy().view(np.uint32)
        for q, t in enumerate(self.assign):
            o, w = int(self.plan.out_offsets[q]), self.shapes[t][1]
            rec = ((a[o:o + w].astype(np.uint64) + b[o:o + w]) & 0xFFFFFFFF).astype(np.uint32)
            if not np.array_equal(rec, self.tables[t][self.alphas[q]].cpu().numpy().view(np.uint32)):
                return False
        return True

    def plan_info(self):
        return {"item_log2": self.item_log2, "items": self.plan.items, "autotune_ms": round(self.tune_ms, 3),
                "graph": True}

    def extras(self):
        # one launch per table (pir_server_eval_device on each table's queries), back to back
        torch, pir, stream = self.torch, self.pir, self.stream
        per = []
        for t in range(len(self.shapes)):
            qs = [q for q, tt in enumerate(self.assign) if tt == t]
            if not qs:
                continue
            kb = pir.pir_key_bytes(self.ns[t])
            keys = torch.frombuffer(bytearray(b"".join(self.pairs[q][0] for q in qs)), dtype=torch.uint8).to(self.device)
            per.append((t, len(qs), keys, torch.empty((len(qs), self.shapes[t][1]), dtype=torch.int32,
                                                      device=self.device)))
            del kb
        def run():
            for t, nq, keys, out in per:
                pir.pir_server_eval_device(self.tables[t], keys, nq, out, stream=stream)
        run()
        torch.cuda.synchronize(self.device)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(3):
            run()
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / 3
        return {"per_table_launches": {"qps": round(self.batch / (ms / 1e3), 2), "ms": round(ms, 4),
                                       "launches": len(per)}}

    def cpu_baseline(self):
        from concurrent.futures import ThreadPoolExecutor

        import oracle

        oracle.build()
        threads = os.cpu_count() or 1
        sample = list(range(0, self.batch, max(1, self.batch // (2 * threads))))[: 2 * threads]
        host = [t.cpu().numpy().view(np.uint32) for t in self.tables]
        t0 = time.perf_counter()
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda q: oracle.answer(self.pairs[q][0], host[self.assign[q]]), sample))
        wall = time.perf_counter() - t0
        return {"value": round(len(sample) / wall, 4), "unit": "queries/s", "cores": min(threads, len(sample)),
                "kind": "oracle", "sample": f"{len(sample)} queries spread over the Zipf mix (oracle FullEval + "
                                            f"inner product), {min(threads, len(sample))} host threads, {wall:.1f} s wall"}


class ServingMix:
    """The serving loop over the 4 resident tables of the serving workload, with
    seeded requests (table uniform, alpha uniform) and both parties' keys."""

    def __init__(self, pir, torch, device, seed, max_count):
        self.pir, self.torch, self.device, self.seed = pir, torch, device, seed
        self.shapes = shapes = wl.SERVING_TABLES
        self.tables = [wl.table_u32_torch(seed * 100 + i, r, w, device) for i, (r, w) in enumerate(shapes)]
        ns = [pir.pir_domain_bits(r) for r, _ in shapes]
        self.srv = pir.Server(max_batch=2048, streams=2)
        self.tids = [self.srv.register_table(t) for t in self.tables]
        self.assign = wl.uniform_tables(seed, len(shapes), max_count)
        rng = np.random.Generator(np.random.PCG64(seed))
        self.alphas = [int(rng.integers(0, shapes[t][0])) for t in self.assign]
        self.pairs = [pir.pir_keygen(ns[t], a, 1, hashlib.sha256(b"serve%d-%d" % (seed, q)).digest())
                      for q, (t, a) in enumerate(zip(self.assign, self.alphas))]
        self.widths = np.array([shapes[t][1] for t in self.assign], np.uint64)
        self.out_off = np.concatenate([[0], np.cumsum(self.widths)[:-1]]).astype(np.uint64)
        self.klens = np.array([len(p[0]) for p in self.pairs], np.uint64)
        self.key_off = np.concatenate([[0], np.cumsum(self.klens)[:-1]]).astype(np.uint64)
        self.keys = (b"".join(p[0] for p in self.pairs), b"".join(p[1] for p in self.pairs))
        self.outs = np.zeros(int(self.widths.sum()), np.uint32)

    def replay(self, rate, count, party=0, outs=None):
        """Poisson arrivals at `rate` queries/s for the first `count` requests:
        per-request latencies (ns) and the elapsed time (s)."""
        arr = wl.poisson_arrivals(self.seed + rate, rate, count)
        return self.srv.replay(arr, [self.tids[t] for t in self.assign[:count]], self.keys[party],
                               self.key_off[:count], self.outs if outs is None else outs, self.out_off[:count])

    def check(self, nchk):
        """Both servers over the first requests reconstruct their rows."""
        outs0, outs1 = np.zeros_like(self.outs), np.zeros_like(self.outs)
        self.replay(2000, nchk, 0, outs0)
        self.replay(2000, nchk, 1, outs1)
        ok = True
        for q in range(nchk):
            o, w = int(self.out_off[q]), int(self.widths[q])
            rec = ((outs0[o:o + w].astype(np.uint64) + outs1[o:o + w]) & 0xFFFFFFFF).astype(np.uint32)
            ok = ok and np.array_equal(rec, self.tables[self.assign[q]][self.alphas[q]].cpu().numpy().view(np.uint32))
        return ok

    def rate_result(self, rate, count):
        """Achieved rate and latency percentiles, overall and per table (the
        tables' work differs 64x, so the overall spread mostly reflects the mix)."""
        lat, el = self.replay(rate, count)
        lat_ms = lat / 1e6
        tabs = np.asarray(self.assign[:count])
        per = {}
        for t, (r, w) in enumerate(self.shapes):
            x = lat_ms[tabs == t]
            if x.size:
                per[f"2^{int(r).bit_length() - 1}x{w}"] = {"p50_ms": round(float(np.percentile(x, 50)), 3),
                                                           "p99_ms": round(float(np.percentile(x, 99)), 3)}
        return {"offered_qps": rate, "requests": count, "achieved_qps": round(count / el, 1),
                "p50_ms": round(float(np.percentile(lat_ms, 50)), 3),
                "p99_ms": round(float(np.percentile(lat_ms, 99)), 3), "per_table": per}

    def plain(self, nq=64):
        """Each query alone in its own launch (pir_server_eval_device), same table mix."""
        torch, pir, device = self.torch, self.pir, self.device
        dk = [torch.frombuffer(bytearray(self.pairs[q][0]), dtype=torch.uint8).to(device) for q in range(nq)]
        po = [torch.empty((1, self.shapes[self.assign[q]][1]), dtype=torch.int32, device=device) for q in range(nq)]
        stream = torch.cuda.current_stream(device)
        for q in range(4):
            pir.pir_server_eval_device(self.tables[self.assign[q]], dk[q], 1, po[q], stream=stream)
        torch.cuda.synchronize(device)
        plain = []
        for q in range(nq):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pir.pir_server_eval_device(self.tables[self.assign[q]], dk[q], 1, po[q], stream=stream)
            b.record(stream)
            b.synchronize()
            plain.append(a.elapsed_time(b))
        return {"qps": round(1e3 / statistics.mean(plain), 2), "p50_ms": round(float(np.percentile(plain, 50)), 4),
                "p99_ms": round(float(np.percentile(plain, 99)), 4), "launches": len(plain)}

    def close(self):
        st = self.srv.stats()
        self.srv.close()
        return st


def run_serving(args):
    """Open-loop Poisson load on the serving loop over 4 resident tables."""
    import torch

    import __graft_entry__ as g

    rank, local_rank, world = dist_env()
    device = torch.device("cuda", local_rank)
    torch.cuda.set_device(device)
    dist_init(world, "nccl")
    g.build()
    import paper_2301_10904_gb300 as pir

    wk = WORKLOADS["serving"]
    seed = rank_seed(wk["seed"], rank)
    rates = [int(x) for x in args.rates.split(",")]
    max_count = max(min(int(r * args.seconds), args.max_requests) for r in rates)
    mix = ServingMix(pir, torch, device, seed, max_count)
    mix.replay(1000, min(200, max_count))  # warm-up (builds lookup tables, allocates the batch buffers)
    ok = mix.check(min(512, max_count))

    results = []
    sampler = ClockSampler(gpu_id_for(device) if rank == 0 else None)
    barrier(world, device)
    with sampler if rank == 0 else _Null():
        for rate in rates:
            results.append(mix.rate_result(rate, min(int(rate * args.seconds), args.max_requests)))
    plain = mix.plain()
    st = mix.close()
    if rank != 0:
        return
    best = max(results, key=lambda r: r["achieved_qps"])
    knee = max([r for r in results if r["achieved_qps"] >= 0.95 * r["offered_qps"]] or [results[0]],
               key=lambda r: r["offered_qps"])
    total_req = sum(r["requests"] for r in results)
    out = {
        "metric": METRIC, "value": best["achieved_qps"], "unit": "queries/s", "n_gpus": world,
        "steps": total_req, "warmup": 200, "ms_per_step": round(1e3 / best["achieved_qps"], 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded SplitMix64 tables, uniform alpha and table, Poisson arrivals, keys from pir_keygen)",
        "config": workload_config("serving", 0, world),
        "server": {"max_batch": 2048, "streams": 2, "max_inflight": st["max_inflight"]},
        "latency_ms": {"p50": knee["p50_ms"], "p99": knee["p99_ms"], "at_offered_qps": knee["offered_qps"]},
        "rates": results,
        "saturation": {"achieved_qps": best["achieved_qps"], "offered_qps": best["offered_qps"],
                       "p50_ms": best["p50_ms"], "p99_ms": best["p99_ms"]},
        "knee_offered_qps": knee["offered_qps"],
        "plain": plain,
        "gpu_launches": st["batches"], "server_stats": st,
        "e2e": {"value": best["achieved_qps"], "unit": "queries/s",
                "h2d_bytes_per_step": int(mix.klens.mean()), "d2h_bytes_per_step": int(mix.widths.mean() * 4),
                "note": "the serving loop is end to end: host keys in, host shares out; per query"},
        "selfcheck_reconstruct_all": ok, "clocks": sampler.summary(),
    }
    print(json.dumps(out), flush=True)


def run_serving_hotfull(args):
    """Hot/full table split (Sec. 4) on the serving loop: every request carries
    exactly Q_hot hot-table and Q_full full-table queries; a request's latency
    is that of its slowest query.  Compared with the same requests sent as
    Q_hot + Q_full full-table queries (no split)."""
    import torch

    import __graft_entry__ as g

    rank, local_rank, world = dist_env()
    device = torch.device("cuda", local_rank)
    torch.cuda.set_device(device)
    dist_init(world, "nccl")
    g.build()
    import paper_2301_10904_gb300 as pir

    wk = WORKLOADS["serving_hotfull"]
    seed = rank_seed(wk["seed"], rank)
    full_rows, width = wl.HOTFULL_FULL
    qh, qf, K = wl.HOTFULL_Q_HOT, wl.HOTFULL_Q_FULL, wl.HOTFULL_WANTED
    q = qh + qf
    z = wl.ZipfRows(seed, full_rows)
    hot_rows = z.top(wl.HOTFULL_HOT_ROWS)
    full = wl.table_u32_torch(seed * 100, full_rows, width, device)
    hot = full[torch.from_numpy(hot_rows.astype(np.int64)).to(device)].contiguous()
    srv = pir.Server(max_batch=2048, streams=2)
    tid_hot, tid_full = srv.register_table(hot), srv.register_table(full)
    rates = [int(x) for x in args.req_rates.split(",")]
    R = max(min(int(r * args.seconds), args.max_requests // q) for r in rates)
    wanted = z.sample(seed + 1, R * K).reshape(R, K)

    def build(split: bool):
        """Per request: keys of both parties, table ids and share offsets of its q queries."""
        k0s, k1s, tids, slots = [], [], [], []
        for r in range(R):
            hk0, hk1, fk0, fk1, slot = pir.pir_hotfull_keygen(
                full_rows, hot_rows, wanted[r], qh if split else 0, qf if split else q,
                seed=hashlib.sha256(b"hotfull%d-%d-%d" % (seed, r, split)).digest())
            nh = qh if split else 0
            hkb = len(hk0) // nh if nh else 0
            fkb = len(fk0) // (q - nh)
            k0s += [hk0[i * hkb:(i + 1) * hkb] for i in range(nh)] + [fk0[i * fkb:(i + 1) * fkb] for i in range(q - nh)]
            k1s += [hk1[i * hkb:(i + 1) * hkb] for i in range(nh)] + [fk1[i * fkb:(i + 1) * fkb] for i in range(q - nh)]
            tids += [tid_hot] * nh + [tid_full] * (q - nh)
            slots.append(slot)
        klens = np.array([len(k) for k in k0s], np.uint64)
        koff = np.concatenate([[0], np.cumsum(klens)[:-1]]).astype(np.uint64)
        ooff = (np.arange(R * q, dtype=np.uint64) * width).astype(np.uint64)
        return b"".join(k0s), b"".join(k1s), np.array(tids, np.uint32), koff, ooff, slots

    plans = {True: build(True), False: build(False)}

    def replay(split, rate, count, party=0):
        keys0, keys1, tids, koff, ooff, _ = plans[split]
        arr = np.repeat(wl.poisson_arrivals(seed + rate, rate, count), q)  # a request's queries arrive together
        outs = np.zeros(count * q * width, np.uint32)
        lat, el = srv.replay(arr, tids[:count * q], keys0 if party == 0 else keys1, koff[:count * q], outs,
                             ooff[:count * q])
        return lat.reshape(count, q).max(axis=1) / 1e6, el, outs

    replay(True, 200, min(50, R))  # warm-up: lookup tables, batch buffers
    # correctness: both servers over the first requests reconstruct every kept row
    nchk = min(64, R)
    ok = True
    for split in (True, False):
        _, _, o0 = replay(split, 400, nchk, 0)
        _, _, o1 = replay(split, 400, nchk, 1)
        rec = ((o0.astype(np.uint64) + o1) & 0xFFFFFFFF).astype(np.uint32).reshape(nchk, q, width)
        for r in range(nchk):
            for i, sl in enumerate(plans[split][5][r]):
                if sl >= 0:
                    ok = ok and np.array_equal(rec[r, sl], full[int(wanted[r, i])].cpu().numpy().view(np.uint32))
    drop = {s: float(np.mean([np.mean(np.asarray(x) < 0) for x in plans[s][5]])) for s in (True, False)}

    results = {True: [], False: []}
    sampler = ClockSampler(gpu_id_for(device) if rank == 0 else None)
    barrier(world, device)
    with sampler if rank == 0 else _Null():
        for split in (True, False):
            for rate in rates:
                count = min(int(rate * args.seconds), R)
                lat, el, _ = replay(split, rate, count)
                results[split].append({"offered_rps": rate, "requests": count, "achieved_rps": round(count / el, 1),
                                       "p50_ms": round(float(np.percentile(lat, 50)), 3),
                                       "p99_ms": round(float(np.percentile(lat, 99)), 3)})
    st = srv.stats()
    srv.close()
    if rank != 0:
        return

    def summary(res):
        best = max(res, key=lambda r: r["achieved_rps"])
        knee = max([r for r in res if r["achieved_rps"] >= 0.95 * r["offered_rps"]] or [res[0]],
                   key=lambda r: r["offered_rps"])
        return best, knee

    best, knee = summary(results[True])
    nbest, nknee = summary(results[False])
    out = {
        "metric": METRIC, "value": round(best["achieved_rps"] * q, 1), "unit": "queries/s", "n_gpus": world,
        "steps": sum(r["requests"] for r in results[True]), "warmup": 50,
        "ms_per_step": round(1e3 / best["achieved_rps"], 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded SplitMix64 table, Zipf(1.1) row popularity through a seeded permutation, "
                "Poisson request arrivals, keys from pir_hotfull_keygen)",
        "config": workload_config("serving_hotfull", 0, world),
        "server": {"max_batch": 2048, "streams": 2, "max_inflight": st["max_inflight"]},
        "latency_ms": {"p50": knee["p50_ms"], "p99": knee["p99_ms"], "at_offered_rps": knee["offered_rps"]},
        "requests_per_s": best["achieved_rps"],
        "rates": results[True],
        "dropped_fraction": round(drop[True], 5),
        "no_split": {"q_full": q, "requests_per_s": nbest["achieved_rps"], "knee_offered_rps": nknee["offered_rps"],
                     "p50_ms": nknee["p50_ms"], "p99_ms": nknee["p99_ms"], "rates": results[False],
                     "dropped_fraction": round(drop[False], 5)},
        "gpu_launches": st["batches"], "server_stats": st,
        "e2e": {"value": round(best["achieved_rps"] * q, 1), "unit": "queries/s",
                "h2d_bytes_per_step": int(len(plans[True][0]) // R), "d2h_bytes_per_step": q * width * 4,
                "note": "the serving loop is end to end: host keys in, host shares out; per request"},
        "selfcheck_reconstruct_all": ok, "clocks": sampler.summary(),
    }
    print(json.dumps(out), flush=True)


class PbrWorkload:
    """Partial batch retrieval (Sec. 4, batch PIR): one table cut into bins, one
    DPF query over each bin per step (pir_pbr_keygen on the client side), every
    bin in one launch (pir_server_eval_pbr).  A query here is one bin's query."""

    def __init__(self, name, wk, pir, torch, device, stream, seed, args):
        self.name, self.pir, self.torch, self.device, self.stream, self.args = name, pir, torch, device, stream, args
        self.rows, self.width, self.bin_rows = wk["rows"], wk["width"], wk["bin_rows"]
        self.desc, self.seed = wk["desc"], seed
        self.prf = PRFS[args.prf]
        self.nbins = -(-self.rows // self.bin_rows)
        self.nb = pir.pir_domain_bits(self.bin_rows)
        self.table = wl.table_u32_torch(seed, self.rows, self.width, device)
        rng = np.random.Generator(np.random.PCG64(seed))
        self.wanted = rng.integers(0, self.rows, self.nbins)  # as many wanted rows as bins: some collide
        k0, k1, self.kept = pir.pir_pbr_keygen(self.rows, self.bin_rows, self.wanted, prf=self.prf,
                                               seed=hashlib.sha256(b"pbr%d" % seed).digest())
        self.keys1 = k1
        self.dkeys = torch.frombuffer(bytearray(k0), dtype=torch.uint8).to(device)
        self.dout = torch.empty((self.nbins, self.width), dtype=torch.int32, device=device)
        self.hkeys = torch.frombuffer(bytearray(k0), dtype=torch.uint8).pin_memory()
        self.hout = torch.empty((self.nbins, self.width), dtype=torch.int32).pin_memory()
        self.dkeys_e2e = torch.empty_like(self.dkeys)
        self.dout_e2e = torch.empty_like(self.dout)
        self.queries_per_step = self.nbins
        self.nodes_per_step = self.nbins * ((1 << self.nb) - 1)
        # a step is one launch of pbr_bfs_scan_kernel: every bin's tree breadth first, then each CTA's
        # own rows of the table.  The roofline is its expansion phase's, the same code and launch shape
        # timed alone through pir_expand_materialise (expand_bfs_kernel); the rest of the step is the
        # row phase, against HBM (see dominant_kernel())
        self.kernel = "pbr_bfs_scan_kernel (expansion phase: expand_bfs_kernel timed alone)"
        self.launches_per_step = 1
        self.scratch = torch.empty((self.nbins, self.bin_rows), dtype=torch.int32, device=device)
        self.h2d_bytes, self.d2h_bytes = len(k0), self.nbins * self.width * 4

    def step(self):
        self.pir.pir_server_eval_pbr(self.table, self.bin_rows, self.dkeys, self.dout, stream=self.stream)

    def dominant_kernel(self, step_ms: float):
        """The expansion alone (CUDA events on the launching stream, 20 launches after 3 warm-up):
        its duration for the roofline, and the rest of the step (the row phase) against HBM."""
        torch = self.torch
        run = lambda: self.pir.pir_expand_materialise(self.bin_rows, self.dkeys, self.nbins, self.scratch,
                                                      stream=self.stream)
        for _ in range(3):
            run()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(self.stream)
        for _ in range(20):
            run()
        b.record(self.stream)
        b.synchronize()
        ms = a.elapsed_time(b) / 20
        scan_ms = max(step_ms - ms, 1e-6)
        scan_bytes = self.rows * self.width * 4  # the table once; the shares stay on chip
        return ms, {"expand_ms": round(ms, 4), "scan_ms_rest_of_step": round(scan_ms, 4),
                    "scan_bytes": scan_bytes, "scan_gbs": round(scan_bytes / (scan_ms / 1e3) / 1e9, 1)}

    def e2e_step(self):
        # pinned host keys in, host shares out: the copies are inside the timed region
        self.dkeys_e2e.copy_(self.hkeys, non_blocking=True)
        self.pir.pir_server_eval_pbr(self.table, self.bin_rows, self.dkeys_e2e, self.dout_e2e, stream=self.stream)
        self.hout.copy_(self.dout_e2e, non_blocking=True)

    def e2e_matches(self):
        self.torch.cuda.synchronize(self.device)
        return bool(np.array_equal(self.hout.numpy(), self.dout.cpu().numpy()))

    def selfcheck(self):
        torch, pir = self.torch, self.pir
        d1 = torch.empty_like(self.dout)
        k1 = torch.frombuffer(bytearray(self.keys1), dtype=torch.uint8).to(self.device)
        pir.pir_server_eval_pbr(self.table, self.bin_rows, k1, d1, stream=self.stream)
        torch.cuda.synchronize(self.device)
        rec = ((self.dout.cpu().numpy().view(np.uint32).astype(np.uint64) + d1.cpu().numpy().view(np.uint32))
               & 0xFFFFFFFF).astype(np.uint32)
        idx = np.asarray(self.wanted, dtype=np.int64)[self.kept]
        want = self.table[torch.from_numpy(idx).to(self.device)].cpu().numpy().view(np.uint32)
        claimed = np.zeros(self.nbins, bool)
        claimed[idx // self.bin_rows] = True
        return bool(np.array_equal(rec[idx // self.bin_rows], want) and not rec[~claimed].any())

    def extras(self):
        return {"pbr": {"wanted_rows_per_step": int(len(self.wanted)), "retrieved_rows_per_step": int(self.kept.sum()),
                        "dropped_fraction": round(1.0 - float(self.kept.sum()) / len(self.wanted), 4),
                        "key_bytes_per_query": self.pir.pir_key_bytes(self.nb)}}

    def cpu_baseline(self):
        import oracle
        from concurrent.futures import ThreadPoolExecutor

        oracle.build()
        threads = os.cpu_count() or 1
        T = self.table.cpu().numpy().view(np.uint32)
        kb = self.pir.pir_key_bytes(self.nb)
        keys = bytes(self.dkeys.cpu().numpy())
        sample = list(range(0, self.nbins, max(1, self.nbins // (8 * threads))))
        t0 = time.perf_counter()
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda b: oracle.answer(keys[b * kb:(b + 1) * kb],
                                                T[b * self.bin_rows:(b + 1) * self.bin_rows]), sample))
        wall = time.perf_counter() - t0
        return {"value": round(len(sample) / wall, 4), "unit": "queries/s", "cores": min(threads, len(sample)),
                "kind": "oracle", "sample": f"{len(sample)} bin queries of this workload (oracle FullEval over the "
                                            f"bin + inner product), {threads} host threads, {wall:.1f} s wall"}


WORKLOAD_CLASSES = {"batched_1m": SingleTableWorkload, "plain_64k": SingleTableWorkload,
                    "large_16m": SingleTableWorkload, "multi_table": MultiTableWorkload, "pbr_1m": PbrWorkload}


def run_ours(args):
    import torch

    import __graft_entry__ as g

    rank, local_rank, world = dist_env()
    device = torch.device("cuda", local_rank)
    torch.cuda.set_device(device)
    dist_init(world, "nccl")
    g.build()
    import paper_2301_10904_gb300 as pir

    wk = WORKLOADS[args.workload]
    stream = torch.cuda.current_stream(device)
    W = WORKLOAD_CLASSES[args.workload](args.workload, wk, pir, torch, device, stream,
                                        rank_seed(wk["seed"], rank), args)

    for _ in range(args.warmup):
        W.step()
    torch.cuda.synchronize(device)
    steps = args.steps  # explicit, or enough for about three seconds of timed work
    if steps is None:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        W.step()
        e1.record(stream)
        torch.cuda.synchronize(device)
        steps = int(min(2000, max(10, 3000.0 / max(e0.elapsed_time(e1), 1e-3))))

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    sampler = ClockSampler(gpu_id_for(device) if rank == 0 else None)
    barrier(world, device)
    torch.cuda.synchronize(device)
    with sampler if rank == 0 else _Null():
        for i in range(steps):
            starts[i].record(stream)
            W.step()
            ends[i].record(stream)
        torch.cuda.synchronize(device)
        barrier(world, device)
    per_step = [s.elapsed_time(e) for s, e in zip(starts, ends)]  # ms
    total_ms = max_over_ranks(starts[0].elapsed_time(ends[-1]), world, device)
    value = W.queries_per_step * world * steps / (total_ms / 1e3)

    selfcheck = W.selfcheck()  # outside the timed region: both servers reconstruct T[alpha]

    # end to end through the public API: pinned host keys in, pinned host shares out
    for _ in range(max(1, min(args.warmup, 3))):
        W.e2e_step()
    e2e_steps = max(3, min(steps, 50))
    e2e_ms = []
    barrier(world, device)
    for _ in range(e2e_steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        W.e2e_step()
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e_total = max_over_ranks(sum(e2e_ms), world, device)
    e2e_ok = W.e2e_matches()
    extras = W.extras()
    if world == 1 and args.other_configs and args.workload == "large_16m":
        extras["other_configs"] = other_configs(args, pir, torch, device, stream)

    if rank != 0:
        return
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    clocks = sampler.summary()
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    kernel_ms = statistics.mean(per_step)
    step_parts = None
    if hasattr(W, "dominant_kernel"):  # a step of several launches: the roofline is its dominant kernel's
        kernel_ms, step_parts = W.dominant_kernel(kernel_ms)
    if getattr(W, "prf", 0) == 1:
        # ChaCha20: the 640 XORs and rotations of 20 rounds per node run on the ALU pipe (64 lanes/clk/SM)
        per_node, unit = CHACHA_ALU_OPS_PER_NODE, "Gop/s"
        peak = sms * 64 * max_mhz * 1e6 / 1e9
        work = f"{CHACHA_ALU_OPS_PER_NODE} ChaCha20 XOR/rotate ops x {W.nodes_per_step} tree nodes per launch"
        basis = f"{sms} SMs x 64 ALU-pipe lanes/clk x {max_mhz:.0f} MHz (derived)"
    else:
        per_node, unit = LOOKUPS_PER_NODE, "Glookup/s"
        peak = sms * 32 * max_mhz * 1e6 / 1e9
        work = (f"{LOOKUPS_PER_NODE} AES table lookups (textbook T-table count; the kernel executes 333 per "
                f"internal node, 311 above leaves) x {W.nodes_per_step} tree nodes per launch")
        basis = f"{sms} SMs x 32 shared-memory lookups/clk x {max_mhz:.0f} MHz (derived)"
    achieved = per_node * W.nodes_per_step / (kernel_ms / 1e3) / 1e9
    cfg = workload_config(args.workload, getattr(W, "prf", 0), world)
    out = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "queries/s",
        "n_gpus": world,
        "steps": steps,
        "warmup": args.warmup,
        "ms_per_step": round(total_ms / steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        # the paper's figure for this workload is with AES-128 keys (Table 4): no ratio for ChaCha20 keys
        "vs_baseline": (round(value / PAPER_QPS[args.workload], 3)
                        if args.workload in PAPER_QPS and getattr(W, "prf", 0) == 0 else None),
        "dtype": "u32",
        "data": "synthetic (seeded SplitMix64 tables, uniform alpha, keys from pir_keygen)",
        "config": cfg,
        **({"plan": W.plan_info()} if hasattr(W, "plan_info") else {}),
        "latency_ms": {"p50": round(float(np.percentile(per_step, 50)), 4),
                       "p99": round(float(np.percentile(per_step, 99)), 4)},
        "gpu_launches": steps * getattr(W, "launches_per_step", 1),
        "roofline": {"bound": "alu", "achieved": round(achieved, 1), "peak": round(peak, 1), "unit": unit,
                     "frac": round(achieved / peak, 4),
                     "traffic": profiled_traffic(args.workload + (":chacha20" if getattr(W, "prf", 0) == 1 else "")),
                     "kernel": W.kernel, "kernel_ms": round(kernel_ms, 4), "work": work, "peak_basis": basis,
                     **({"step_parts": step_parts} if step_parts else {})},
        "e2e": {"value": round(W.queries_per_step * world * e2e_steps / (e2e_total / 1e3), 2), "unit": "queries/s",
                "h2d_bytes_per_step": W.h2d_bytes, "d2h_bytes_per_step": W.d2h_bytes,
                "p50_ms": round(float(np.percentile(e2e_ms, 50)), 4), "bit_exact_vs_device": e2e_ok},
        "selfcheck_reconstruct_all": selfcheck,
        "clocks": clocks,
    }
    out.update(extras)
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = W.cpu_baseline()
    print(json.dumps(out), flush=True)


def _events_ms(torch, stream, fn, reps):
    """Total device time of `reps` back-to-back calls, CUDA events on the launching stream."""
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b)


def other_configs(args, pir, torch, device, stream):
    """Compact measurements of the four other workload configurations, run in
    the headline run's process after its timed region: the plain single query
    (2^16 x 16), the batched table (2^20 x 64, 256 queries), the 8-table Zipf
    mix (graph replay) and the serving loop at one offered rate below its knee
    and one above.  Each reports its own bit-exact reconstruction check."""
    out = {}
    wk = WORKLOADS["plain_64k"]
    P = SingleTableWorkload("plain_64k", wk, pir, torch, device, stream, wk["seed"], args)
    for _ in range(10):
        P.step()
    torch.cuda.synchronize(device)
    lat = []
    for _ in range(100):
        lat.append(_events_ms(torch, stream, P.step, 1))
    back = _events_ms(torch, stream, P.step, 200) / 200
    for _ in range(5):
        P.e2e_step()
    e2e = _events_ms(torch, stream, P.e2e_step, 200) / 200
    out["plain_64k"] = {"workload": wk["desc"], "device_us_per_query": round(back * 1e3, 2),
                        "qps": round(1e3 / back, 1), "p50_us": round(float(np.percentile(lat, 50)) * 1e3, 2),
                        "p99_us": round(float(np.percentile(lat, 99)) * 1e3, 2),
                        "e2e_qps": round(1e3 / e2e, 1), "e2e_us_per_query": round(e2e * 1e3, 2),
                        "e2e_note": "pir_server_eval: pinned host key in, pinned host share out, one call per query",
                        "plan": P.plan_info(), "selfcheck_reconstruct_all": P.selfcheck(),
                        "e2e_bit_exact_vs_device": P.e2e_matches()}
    del P
    wk = WORKLOADS["batched_1m"]
    B = SingleTableWorkload("batched_1m", wk, pir, torch, device, stream, wk["seed"], args)
    for _ in range(3):
        B.step()
    ms = _events_ms(torch, stream, B.step, 10) / 10
    qps = B.batch / (ms / 1e3)
    out["batched_1m"] = {"workload": wk["desc"], "qps": round(qps, 1), "ms_per_step": round(ms, 4),
                         "vs_paper_table4": round(qps / PAPER_QPS["batched_1m"], 2),
                         "plan": B.plan_info(), "selfcheck_reconstruct_all": B.selfcheck()}
    del B
    wk = WORKLOADS["multi_table"]
    M = MultiTableWorkload("multi_table", wk, pir, torch, device, stream, wk["seed"], args)
    for _ in range(3):
        M.step()
    ms = _events_ms(torch, stream, M.step, 10) / 10
    out["multi_table"] = {"workload": wk["desc"], "qps": round(M.batch / (ms / 1e3), 1), "ms_per_step": round(ms, 4),
                          "plan": M.plan_info(), "selfcheck_reconstruct_all": M.selfcheck()}
    del M
    wk = WORKLOADS["serving"]
    rates = (2000, 8000)
    mix = ServingMix(pir, torch, device, wk["seed"], 4000)
    mix.replay(1000, 200)
    ok = mix.check(256)
    res = [mix.rate_result(2000, 2000), mix.rate_result(8000, 4000)]
    plain = mix.plain(32)
    st = mix.close()
    out["serving"] = {"workload": wk["desc"], "rates": res, "plain": plain, "batches": st["batches"],
                      "note": f"offered {rates[0]} queries/s is below the saturation knee, {rates[1]} above it",
                      "selfcheck_reconstruct_all": ok}
    torch.cuda.synchronize(device)
    return out


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


# ----------------------------------------------------------------------------- reference arm (the oracle)

def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    wk = WORKLOADS[args.workload]
    steps, warm = args.steps or 5, args.warmup
    if args.workload in ("multi_table", "serving"):
        # the same query mix over the same tables; each step a bounded sample of its queries
        if args.workload == "multi_table":
            shapes = list(zip(wl.MULTI_TABLE_ROWS, wl.MULTI_TABLE_WIDTHS))
            assign = wl.zipf_assignment(wk["seed"], len(shapes), wl.MULTI_TABLE_QUERIES)
        else:
            shapes = wl.SERVING_TABLES
            assign = wl.uniform_tables(wk["seed"], len(shapes), 4096)
        tables = [wl.table_u32(wk["seed"] * 100 + i, r, w) for i, (r, w) in enumerate(shapes)]

        def one_step(i):
            from concurrent.futures import ThreadPoolExecutor

            import oracle

            threads = os.cpu_count() or 1
            per = threads if args.workload == "serving" else 2 * threads  # serving queries average 5.6M leaves
            qs = [(i * per + j) % len(assign) for j in range(per)]
            keys = []
            for q in qs:
                t = assign[q]
                n = wl.domain_bits(shapes[t][0])
                r0, r1, c0 = wl.key_randomness(wk["seed"] + q, n, 1)[0]
                keys.append((t, oracle.gen(n, q % shapes[t][0], 1, r0, r1, c0)[0]))
            t0 = time.perf_counter()
            with ThreadPoolExecutor(threads) as ex:
                list(ex.map(lambda tk: oracle.answer(tk[1], tables[tk[0]]), keys))
            return len(qs) / (time.perf_counter() - t0), threads, len(qs), time.perf_counter() - t0
        rows = width = None
    elif args.workload == "serving_hotfull":
        # one request per step: its Q_hot hot-table and Q_full full-table queries (oracle keys)
        full_rows, width = wl.HOTFULL_FULL
        rows = full_rows
        z = wl.ZipfRows(wk["seed"], full_rows)
        hot_rows = z.top(wl.HOTFULL_HOT_ROWS)
        full_np = wl.table_u32(wk["seed"] * 100, full_rows, width)
        hot_np = np.ascontiguousarray(full_np[hot_rows.astype(np.int64)])
        nh, nf = wl.domain_bits(hot_rows.size), wl.domain_bits(full_rows)

        def one_step(i):
            from concurrent.futures import ThreadPoolExecutor

            import oracle

            threads = os.cpu_count() or 1
            wanted = z.sample(wk["seed"] + 1 + i, wl.HOTFULL_WANTED)
            ha, hb, fa, fb, _ = oracle.hotfull_plan(full_rows, hot_rows, wanted, wl.HOTFULL_Q_HOT,
                                                    wl.HOTFULL_Q_FULL)
            jobs = []
            for s_, (a, b) in enumerate(zip(ha, hb)):
                r0, r1, c0 = wl.key_randomness(wk["seed"] + 31 * i + s_, nh, 1)[0]
                jobs.append((hot_np, oracle.gen(nh, a, b, r0, r1, c0)[0]))
            for s_, (a, b) in enumerate(zip(fa, fb)):
                r0, r1, c0 = wl.key_randomness(wk["seed"] + 31 * i + 100 + s_, nf, 1)[0]
                jobs.append((full_np, oracle.gen(nf, a, b, r0, r1, c0)[0]))
            t0 = time.perf_counter()
            with ThreadPoolExecutor(threads) as ex:
                list(ex.map(lambda tk: oracle.answer(tk[1], tk[0]), jobs))
            wall = time.perf_counter() - t0
            return len(jobs) / wall, min(threads, len(jobs)), len(jobs), wall
    elif args.workload == "pbr_1m":
        rows, width, bin_rows = wk["rows"], wk["width"], wk["bin_rows"]
        table_np = wl.table_u32(wk["seed"], rows, width)
        nb = wl.domain_bits(bin_rows)
        nbins = -(-rows // bin_rows)

        def one_step(i):
            from concurrent.futures import ThreadPoolExecutor

            import oracle

            threads = os.cpu_count() or 1
            bins = [(i * 16 * threads + j) % nbins for j in range(16 * threads)]
            keys = []
            for b in bins:
                r0, r1, c0 = wl.key_randomness(wk["seed"] + b, nb, 1)[0]
                keys.append((b, oracle.gen(nb, b % bin_rows, 1, r0, r1, c0)[0]))
            t0 = time.perf_counter()
            with ThreadPoolExecutor(threads) as ex:
                list(ex.map(lambda bk: oracle.answer(bk[1], table_np[bk[0] * bin_rows:(bk[0] + 1) * bin_rows]),
                            keys))
            return len(bins) / (time.perf_counter() - t0), threads, len(bins), time.perf_counter() - t0
    else:
        rows, width = wk["rows"], wk["width"]
        table_np = wl.table_u32(wk["seed"], rows, width)

        def one_step(i, quick=False):
            return oracle_qps(rows, width, wk["seed"] + i, table_np, target_cpu_s=2.0 if quick else 4.0)
    for i in range(warm):
        one_step(i)
    times, queries, cores = [], 0, 1
    for i in range(steps):
        qps, cores, nq, wall = one_step(warm + i)
        times.append(wall)
        queries += nq
    total = sum(times)
    value = queries / total
    out = {
        "impl": "reference",
        "metric": METRIC, "value": round(value, 4), "unit": "queries/s", "n_gpus": world, "steps": steps,
        "warmup": warm, "ms_per_step": round(1e3 * total / steps, 2), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload_config(args.workload, 0, world),
        "cpu_baseline": {"value": round(value, 4), "unit": "queries/s", "cores": cores, "kind": "oracle",
                         "sample": f"{queries // steps} queries per step (oracle FullEval + inner product; "
                                   f"a query longer than the step is cut into row ranges over the threads), "
                                   f"{cores} host threads"},
        "e2e": {"value": round(value, 4), "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="large_16m")
    ap.add_argument("--prf", choices=sorted(PRFS), default="aes128",
                    help="PRF of the keys (single-table workloads): AES-128 or ChaCha20 (Sec. 3.2.6, Table 5)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rates", default="1000,2000,4000,6000,10000,20000,50000,100000,200000",
                    help="serving workload: offered Poisson rates (queries/s)")
    ap.add_argument("--req-rates", default="100,200,400,800,1200,1600,2400,4000",
                    help="hot/full serving workload: offered Poisson request rates (requests/s)")
    ap.add_argument("--seconds", type=float, default=1.0, help="serving workload: arrival span per rate")
    ap.add_argument("--max-requests", type=int, default=8000, help="serving workload: requests per rate, at most")
    ap.add_argument("--no-materialised", dest="materialised", action="store_false",
                    help="skip the materialised (share matrix in HBM) comparison leg")
    ap.add_argument("--no-other-configs", dest="other_configs", action="store_false",
                    help="large_16m at N=1: skip the compact runs of the other four configurations")
    ap.add_argument("--no-scan", dest="scan", action="store_false",
                    help="skip the streaming-scan (HBM roofline) leg on tables larger than L2")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "serving_hotfull":
        run_serving_hotfull(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
