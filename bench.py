#!/usr/bin/env python
"""Benchmark of the compressed-domain query path on one GB300 (or N replicas).

Workload (default): the heterogeneous 100M-row table -- int32 RLE key (mean
run 1000), 10,000-entry dictionary column with Zipf(1.1) codes packed in 14
bits, 1%-dense index-encoded int64, plain int32, 20-bit bit-packed int64 --
and SELECT c1, c2, SUM(c3), SUM(c5), MIN(c5), MAX(c5), COUNT(*) WHERE c2 IN
(64 strings) AND c4 BETWEEN 250000 AND 749999 GROUP BY c1, c2.

One step = one query (plan, init, fused kernel, finalize) over the table
resident in HBM.  The inputs (838 MB compressed) are larger than the 129 MB
L2, so no flush is needed between steps.  Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "logical rows/s"
UNIT = "rows/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="cq", choices=["cq", "reference"])
    ap.add_argument("--workload", default="heterogeneous",
                    choices=["heterogeneous", "tiny", "nested", "batched", "serving", "runsweep"])
    ap.add_argument("--rates", default="100,500,1000,2000,5000", help="serving: arrival rates (queries/s)")
    ap.add_argument("--serve-seconds", type=float, default=3.0, help="serving: measured arrivals per rate and mode")
    ap.add_argument("--serve-warmup", type=float, default=1.0,
                    help="serving: seconds of arrivals before the measured ones (latencies not counted)")
    ap.add_argument("--serve-modes", default="batched,one_at_a_time,decompress_then_scan")
    ap.add_argument("--queries", type=int, default=4096, help="batched: queries per batch")
    ap.add_argument("--parts", type=int, default=256, help="batched: partitions in the pool")
    ap.add_argument("--part-max", type=float, default=5e7, help="batched: largest partition (rows)")
    ap.add_argument("--dts-sample", type=int, default=128,
                    help="batched: queries timed on the decompress-then-scan path")
    ap.add_argument("--rows", type=int, default=0, help="override the workload's row count")
    ap.add_argument("--seed", type=int, default=20250611)
    ap.add_argument("--mode", default="fused", choices=["fused", "decompress_then_scan"])
    ap.add_argument("--tile-rows", type=int, default=0)
    ap.add_argument("--stages", type=int, default=0)
    ap.add_argument("--table-slots", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="heterogeneous workload: skip the decompress-then-scan comparison and the 20e9-row "
                         "nested query reported beside the main line")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def workload(args):
    from paper_2506_10092_gb300 import datagen as dg
    if args.workload == "tiny":
        n = args.rows or 1_000_000
        table, plan = dg.tiny_two_rle(n, seed=args.seed)
        name = f"tiny-two-rle-{n}"
    elif args.workload == "nested":
        # generated in device memory by run_cq (too large for the host)
        n = args.rows or 20_000_000_000
        return f"nested-lean-{n}", None, dg.nested_plan(lean=True)
    else:
        n = args.rows or 100_000_000
        table, plan = dg.heterogeneous(n, seed=args.seed)
        name = f"heterogeneous-5col-{n}"
    return name, table, plan


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# the device code of the shape-specialised row kernel (compiled at run time
# from these headers and the shape class cq_jit.cu writes)
ROW_KERNEL_SOURCES = ("cq_fast.cuh", "cq_rowpath.cuh", "cq_phases.cuh", "cq_device.cuh", "cq_desc.h", "cq_jit.cu")


def _code_only(text: str) -> str:
    """Source text without comments and whitespace (comment edits keep the hash)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return re.sub(r"\s+", "", text)


def kernel_source_hash(read=None) -> str:
    h = hashlib.sha256()
    for name in ROW_KERNEL_SOURCES:
        if read is None:
            with open(os.path.join(ROOT, "paper_2506_10092_gb300", "csrc", name)) as fh:
                text = fh.read()
        else:
            text = read(name)
        h.update(_code_only(text).encode())
    return h.hexdigest()[:16]


def profile_traffic(workload_name: str, n_rows: int = 0):
    """dram bytes per launch of the fused kernel from a committed ncu summary
    (profiles/*.json) taken on the current kernel sources, else None.  A
    summary names its workload (bytes per launch as captured and scaled) or a
    workload family whose traffic grows with the rows (bytes scaled from the
    captured rows to n_rows)."""
    import glob
    h = kernel_source_hash()
    for p in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.json"))):
        try:
            with open(p) as f:
                d = json.load(f)
            if d.get("kernel_sources_sha256_16") != h:
                continue
            if d.get("workload") == workload_name:
                return float(d["dram_bytes_per_launch"])
            fam = d.get("family")
            if fam and workload_name.startswith(fam) and n_rows and d.get("capture_rows"):
                cap = float(d["dram_bytes_read_capture"]) + float(d["dram_bytes_write_capture"])
                return cap * n_rows / float(d["capture_rows"])
        except Exception:
            continue
    return None


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float) -> float:
    """The largest value of x over all ranks (the job's time is its slowest
    rank's); x itself with one process."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return x
    dev = "cuda" if tdist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def exec_opts(cq, args):
    mode = cq.CQ_EXEC_FUSED if args.mode == "fused" else cq.CQ_EXEC_DECOMPRESS_THEN_SCAN
    return cq.exec_options(mode=mode, tile_rows=args.tile_rows, stages=args.stages, table_slots=args.table_slots,
                           ctas_per_sm=args.ctas_per_sm)


def cpu_oracle_rate(table, plan, seconds: float):
    """The oracle as it stands, on this host's cores, over a bounded prefix
    sample of the workload.  Returns (rows/s, cores, sample description)."""
    from oracle import oracle
    cores = oracle.cores()
    probe = min(table.n_rows, 2_000_000)
    t0 = time.perf_counter()
    oracle.query(table, plan, row_ranges=[(0, probe)], n_threads=cores)
    dt = max(1e-3, time.perf_counter() - t0)
    rows = int(min(table.n_rows, max(probe, probe * seconds / dt)))
    t0 = time.perf_counter()
    oracle.query(table, plan, row_ranges=[(0, rows)], n_threads=cores)
    dt = time.perf_counter() - t0
    return rows / dt, cores, f"first {rows} rows of the same table, {cores} threads, {dt:.1f} s"


def run_reference(args):
    from paper_2506_10092_gb300 import datagen as dg
    ws, rank, _ = dist()
    if rank != 0:
        return
    if args.workload in ("batched", "serving"):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times single queries (heterogeneous, "
                                                             "tiny, nested); it has no batched or serving form"}),
              flush=True)
        return
    name, table, plan = workload(args)
    if table is None:
        # the nested table has no host copy at full size: time a same-shape sample
        table, plan = dg.nested(min(args.rows or 20_000_000_000, 20_000_000), seed=args.seed, lean=True)
    from oracle import oracle
    cores = oracle.cores()
    probe = min(table.n_rows, 1_000_000)
    t0 = time.perf_counter()
    oracle.query(table, plan, row_ranges=[(0, probe)], n_threads=cores)
    rate = probe / max(1e-3, time.perf_counter() - t0)
    budget = 90.0 / max(1, args.steps + args.warmup)      # seconds per step
    rows = int(min(table.n_rows, max(100_000, rate * budget)))
    for _ in range(args.warmup):
        oracle.query(table, plan, row_ranges=[(0, rows)], n_threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.query(table, plan, row_ranges=[(0, rows)], n_threads=cores)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = rows * args.steps / total
    sample = f"first {rows} rows per step of the same table, {cores} threads"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": name, "rows": table.n_rows, "sample_rows": rows},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def pinned_copy(torch, a):
    import numpy as np
    t = torch.empty(a.shape[0], dtype=getattr(torch, str(a.dtype)) if str(a.dtype) != "uint32" else torch.int32,
                    pin_memory=True)
    t.numpy()[:] = a.view(np.int32) if str(a.dtype) == "uint32" else a
    return t


def run_cq(args):
    import numpy as np
    import torch
    from paper_2506_10092_gb300 import cq
    from paper_2506_10092_gb300 import datagen as dg

    ws, rank, local = dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    name, table, plan = workload(args)
    used = dg.plan_columns(plan)
    ctx = cq.cq_ctx_create(local, stream)
    dn = None
    if table is None:
        # nested table: RLE runs from the host, per-row columns generated on the device
        from paper_2506_10092_gb300 import devgen
        n_rows = args.rows or 20_000_000_000
        t_gen = time.perf_counter()
        dn = devgen.DeviceNested(cq, ctx, n_rows, seed=args.seed)
        torch.cuda.synchronize()
        t_gen = time.perf_counter() - t_gen
        t = dn.table
        alg_bytes = dn.query_bytes(plan)
    else:
        n_rows = table.n_rows
        alg_bytes = dg.compressed_bytes(table, used)
        t, cols = cq.table_from(ctx, table)
    ps = cq.PlanStruct(plan)
    opts = exec_opts(cq, args)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # warm-up
    for _ in range(max(3, args.warmup)):
        r = cq.cq_query_run(t, ps, stream=stream, opts=opts)
        cq.cq_result_wait(r)
        r.close()
    n_groups = None
    clocks = Clocks(local)
    torch.cuda.synchronize()
    barrier()
    clocks.start()
    time.sleep(0.2)
    results = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        results.append(cq.cq_query_run(t, ps, stream=stream, opts=opts))
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    kernel_us = [cq.cq_result_kernel_time_us(r) for r in results]
    n_groups = cq.cq_result_num_groups(results[-1])
    for r in results:
        cq.cq_result_wait(r)
        r.close()
    elapsed_ms = max_over_ranks(elapsed_ms)
    ms_per_step = elapsed_ms / args.steps
    value = n_rows * args.steps * ws / (elapsed_ms / 1000.0)
    k_us = statistics.mean(kernel_us)
    peak, peak_src = measured_peak()
    achieved = alg_bytes / (k_us * 1e-6) / 1e9
    traffic = profile_traffic(name, n_rows)

    # end to end through the public API: pinned host buffers -> columns ->
    # query -> result read back, every step
    e2e = None
    if dn is not None:
        e2e = {"value": None, "unit": UNIT, "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
               "note": "per-row columns are generated in device memory; the table has no host copy"}
    elif not args.no_e2e:
        host = []
        h2d = 0
        for c in table.columns:
            if c.enc == "rle":
                host.append((c, pinned_copy(torch, c.run_values), pinned_copy(torch, c.run_ends)))
                h2d += c.run_values.nbytes + c.run_ends.nbytes
            elif c.enc in ("dict", "packed"):
                need = (c.n_rows * c.bit_width + 31) // 32
                host.append((c, pinned_copy(torch, c.words[:((need + 3) // 4) * 4 + 4]), None))
                h2d += need * 4
            elif c.enc == "index":
                host.append((c, pinned_copy(torch, c.values), pinned_copy(torch, c.positions)))
                h2d += c.values.nbytes + c.positions.nbytes
            else:
                host.append((c, pinned_copy(torch, c.values), None))
                h2d += c.values.nbytes

        def e2e_step():
            hc = []
            for c, a, b in host:
                if c.enc == "rle":
                    hc.append(cq.cq_column_create_rle(ctx, a, b, c.n_rows))
                elif c.enc == "dict":
                    hc.append(cq.cq_column_create_dict(ctx, c.strings, a, c.bit_width, c.n_rows))
                elif c.enc == "packed":
                    hc.append(cq.cq_column_create_bitpacked(ctx, a, c.bit_width, c.base, c.n_rows))
                elif c.enc == "index":
                    hc.append(cq.cq_column_create_index(ctx, a, b, c.default, c.n_rows))
                else:
                    hc.append(cq.cq_column_create_plain(ctx, a))
            tb = cq.cq_table_bind(ctx, hc)
            res = cq.cq_query_run(tb, ps, stream=stream, opts=opts)
            out = cq.fetch_all(res)
            res.close()
            tb.close()
            for h in hc:
                h.close()
            return sum(o.nbytes for o in out)

        e2e_step()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(args.e2e_steps):
            d2h = e2e_step()
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": table.n_rows * args.e2e_steps * ws / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h + 16, "steps": args.e2e_steps,
               "note": "columns created from pinned host buffers (library copy + validation), query, result fetch"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        sample_table = table
        if dn is not None:
            sample_table = dg.nested_subtable(dn.runs, args.seed, [(0, min(n_rows, 20_000_000))])
        rate, cores, sample = cpu_oracle_rate(sample_table, plan, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": name, "rows": n_rows, "compressed_bytes": alg_bytes, "groups": n_groups,
                       "mode": args.mode, "parallelism": f"replicas{ws}",
                       "l2": "inputs larger than L2 (compressed columns exceed 129 MB); no flush"},
            "compressed_gbs": alg_bytes * args.steps * ws / (elapsed_ms / 1000.0) / 1e9,
            "pct_hbm_peak": alg_bytes * args.steps / (elapsed_ms / 1000.0) / 1e9 / peak,
            "kernel_us": k_us,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "cq_row_jit (row kernel specialised to the query shape)"
                         if dn is not None or args.workload != "tiny" else "seg_query_kernel",
                         "peak_source": f"{peak_src} hbm_gbs",
                         "algorithmic_bytes_per_launch": alg_bytes},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": launches_per_query(n_rows) * args.steps,
        }
        if args.workload == "heterogeneous" and args.mode == "fused" and not args.no_secondary:
            line["decompress_then_scan"] = run_dts_comparison(cq, t, ps, stream, n_rows, ms_per_step, torch)
            del t, cols
            torch.cuda.synchronize()
            line["nested_20e9"] = run_nested_secondary(cq, ctx, stream, args, torch, peak)
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def launches_per_query(n_rows: int) -> int:
    """Kernels one fused query launches: init, the fused kernel (one launch per
    2^31 rows, a SUM fold between two), three finalize kernels."""
    parts = max(1, -(-n_rows // (1 << 31)))
    return 1 + parts + (parts - 1) + 3


def run_dts_comparison(cq, t, ps, stream, n_rows, fused_ms, torch, steps: int = 3):
    """The same query on the decompress-then-scan comparison path (expand every
    referenced column to flat int64 arrays, then scan them), timed on the same
    GPU; steps after one warm-up."""
    opts = cq.exec_options(mode=cq.CQ_EXEC_DECOMPRESS_THEN_SCAN)
    r = cq.cq_query_run(t, ps, stream=stream, opts=opts)
    cq.cq_result_wait(r)
    r.close()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    res = [cq.cq_query_run(t, ps, stream=stream, opts=opts) for _ in range(steps)]
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    for r in res:
        cq.cq_result_wait(r)
        r.close()
    return {"ms_per_step": ms, "rows_per_s": n_rows / (ms / 1000.0), "steps": steps,
            "fused_speedup": ms / fused_ms,
            "note": "every referenced column expanded to flat int64 on the device, then the row scan"}


def run_nested_secondary(cq, ctx, stream, args, torch, peak, steps: int = 3):
    """The largest single-GPU configuration beside the main line: the 20e9-row
    nested table (62.4 GB of compressed columns resident), its c3-range query
    GROUP BY c2, c4; device time of the fused kernel and of the whole query."""
    from paper_2506_10092_gb300 import datagen as dg
    from paper_2506_10092_gb300 import devgen
    try:
        n_rows = 20_000_000_000
        t_gen = time.perf_counter()
        dn = devgen.DeviceNested(cq, ctx, n_rows, seed=args.seed)
        torch.cuda.synchronize()
        t_gen = time.perf_counter() - t_gen
        plan = dg.nested_plan(lean=True)
        ps = cq.PlanStruct(plan)
        alg = dn.query_bytes(plan)
        for _ in range(2):
            r = cq.cq_query_run(dn.table, ps, stream=stream)
            cq.cq_result_wait(r)
            r.close()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        res = [cq.cq_query_run(dn.table, ps, stream=stream) for _ in range(steps)]
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        k_us = statistics.mean(cq.cq_result_kernel_time_us(r) for r in res)
        groups = cq.cq_result_num_groups(res[-1])
        for r in res:
            r.close()
        del dn
        torch.cuda.synchronize()
        return {"workload": f"nested-lean-{n_rows}", "rows": n_rows, "ms_per_step": ms,
                "rows_per_s": n_rows / (ms / 1000.0), "compressed_bytes": alg, "groups": groups,
                "kernel_us": k_us, "achieved_gbs": alg / (k_us * 1e-6) / 1e9,
                "frac_of_measured_hbm": alg / (k_us * 1e-6) / 1e9 / peak, "steps": steps,
                "table_build_s": t_gen, "launches_per_query": launches_per_query(n_rows),
                # DRAM bytes of the whole query (all launches), scaled from the
                # committed ncu summary of the same kernel, or None
                "traffic_per_query": profile_traffic(f"nested-lean-{n_rows}", n_rows)}
    except Exception as e:   # the main line stands without it
        return {"workload": "nested-lean-20000000000", "error": str(e)[:300]}


# ---------------------------------------------------------------- run-length sweep
def run_runsweep(args):
    """Compressed GB/s of pure run-length queries as the runs lengthen: the
    two-RLE template (A < 50 GROUP BY B) over 100M rows at mean runs 8 / 5,
    1e3 and 1e5, and a c3-range query GROUP BY c2 over the RLE columns of a
    1e9-row nested table.  Segment-mode work follows the runs, so the
    compressed GB/s should not fall as runs lengthen."""
    import torch
    from paper_2506_10092_gb300 import cq
    from paper_2506_10092_gb300 import datagen as dg
    from paper_2506_10092_gb300 import devgen
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    ctx = cq.cq_ctx_create(0, stream)
    n = args.rows or 100_000_000
    rows_out = []

    def timed(t, ps, n_rows, alg, label, kernel=0):
        opts = cq.exec_options(kernel=kernel)
        for _ in range(max(3, args.warmup)):
            r = cq.cq_query_run(t, ps, stream=stream, opts=opts)
            cq.cq_result_wait(r)
            r.close()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        res = [cq.cq_query_run(t, ps, stream=stream, opts=opts) for _ in range(args.steps)]
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1) / args.steps
        k_us = statistics.mean(cq.cq_result_kernel_time_us(r) for r in res)
        for r in res:
            r.close()
        walk = {0: "planner's choice", 2: "tiles", 3: "runs"}[kernel]
        rows_out.append({"case": label, "walk": walk, "rows": n_rows, "compressed_bytes": alg, "ms_per_step": ms,
                         "kernel_us": k_us, "rows_per_s": n_rows / (ms / 1e3),
                         "compressed_gbs_kernel": alg / (k_us * 1e-6) / 1e9})
        print(json.dumps(rows_out[-1]), file=sys.stderr, flush=True)

    for ma, mb in ((8.0, 5.0), (1e3, 625.0), (1e5, 62500.0)):
        table, plan = dg.tiny_two_rle(n, seed=args.seed, mean_a=ma, mean_b=mb)
        t, cols = cq.table_from(ctx, table)
        for kernel in (2, 3, 0):
            timed(t, cq.PlanStruct(plan), n, dg.compressed_bytes(table, dg.plan_columns(plan)),
                  f"two-RLE mean runs {ma:g}/{mb:g}", kernel)
        del t, cols, table
    dn = devgen.DeviceNested(cq, ctx, 1_000_000_000, seed=args.seed)
    plan = dg.Plan([dg.Pred(2, "between", 200, 699)], [1], [dg.Agg("count"), dg.Agg("sum", 2), dg.Agg("max", 0)])
    for kernel in (2, 3, 0):
        timed(dn.table, cq.PlanStruct(plan), dn.n_rows, dn.query_bytes(plan), "nested c1..c3 RLE, 1e9 rows", kernel)
    print(json.dumps({"metric": "compressed GB/s of pure run-length queries", "value": None, "unit": "GB/s",
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                      "config": {"workload": "run-length sweep", "parallelism": "replicas1"},
                      "by_case": rows_out, "gpu_launches": 5 * args.steps * len(rows_out)}), flush=True)


# ---------------------------------------------------------------- batched workload
def _tiny_part(n, seed):
    from paper_2506_10092_gb300 import datagen as dg
    t, _ = dg.tiny_two_rle(int(n), seed=int(seed))
    return t


def build_pool(args, cq, ctx, torch):
    """The partition pool of the batched workload: sizes log-uniform in
    [1e4, part_max]; each partition holds the two-RLE table (drawn on the host
    by a spawn process pool) and the nested table (RLE runs on the host,
    per-row columns generated on the device)."""
    import multiprocessing as mp
    import numpy as np
    from paper_2506_10092_gb300 import datagen as dg
    from paper_2506_10092_gb300 import devgen
    rng = np.random.default_rng([args.seed, 4])
    sizes = dg.partition_sizes(rng, args.parts, 1e4, args.part_max)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        tiny = pool.starmap(_tiny_part, [(int(n), args.seed + 1000 + i) for i, n in enumerate(sizes)])
    parts = []
    for i, n in enumerate(sizes):
        th, tcols = cq.table_from(ctx, tiny[i], device=True)
        nest = devgen.DeviceNested(cq, ctx, int(n), seed=args.seed + 2000 + i)
        parts.append({"n": int(n), "tiny": (tiny[i], th, tcols), "nested": nest})
    torch.cuda.synchronize()
    return sizes, parts


def query_bytes(part, kind, plan):
    """Compressed bytes the query reads (its referenced columns)."""
    from paper_2506_10092_gb300 import datagen as dg
    if kind == "tiny":
        return dg.compressed_bytes(part["tiny"][0], dg.plan_columns(plan))
    return part["nested"].query_bytes(plan)


def run_batched(args):
    import numpy as np
    import torch
    from paper_2506_10092_gb300 import cq
    from paper_2506_10092_gb300 import datagen as dg

    ws, rank, local = dist()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    ctx = cq.cq_ctx_create(local, stream)
    t_gen = time.perf_counter()
    sizes, parts = build_pool(args, cq, ctx, torch)
    t_gen = time.perf_counter() - t_gen
    rng = np.random.default_rng([args.seed, 5])
    qs = dg.batch_queries(rng, args.queries, len(parts), lean=True)
    handles, plans, rows, nbytes = [], [], 0, 0
    for part_i, kind, plan in qs:
        part = parts[part_i]
        handles.append(part["tiny"][1] if kind == "tiny" else part["nested"].table)
        plans.append(cq.PlanStruct(plan))
        rows += part["n"]
        nbytes += query_bytes(part, kind, plan)
    torch.cuda.synchronize()

    # autotune the batch shape, then time batches with the tuned shape
    best, tuned_us = cq.cq_batch_tune(handles, plans, stream=stream)

    def batch_step():
        return cq.cq_batch_run(handles, plans, stream=stream)

    for _ in range(max(3, args.warmup)):
        for r in batch_step():
            r.close()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.2)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    held = []
    t_host = time.perf_counter()
    ev0.record(stream)
    for _ in range(args.steps):
        held.append(batch_step())
    ev1.record(stream)
    ev1.synchronize()
    t_host = time.perf_counter() - t_host
    clk = clocks.stop()
    elapsed = ev0.elapsed_time(ev1) / 1000.0
    launch_us = [cq.cq_result_device_time_us(h[0]) for h in held]
    for h in held:
        for r in h:
            r.close()
    held = None
    peak, peak_src = measured_peak()

    # one query at a time: the same queries, one cq_query_run each
    ev0.record(stream)
    solo = [cq.cq_query_run(h, p, stream=stream) for h, p in zip(handles, plans)]
    ev1.record(stream)
    ev1.synchronize()
    solo_s = ev0.elapsed_time(ev1) / 1000.0
    for r in solo:
        r.close()

    # decompress-then-scan on a sample of the queries
    n_dts = min(args.dts_sample, len(handles))
    dts_opts = cq.exec_options(mode=cq.CQ_EXEC_DECOMPRESS_THEN_SCAN)
    dts_rows = sum(parts[q[0]]["n"] for q in qs[:n_dts])
    ev0.record(stream)
    dts = [cq.cq_query_run(handles[i], plans[i], stream=stream, opts=dts_opts) for i in range(n_dts)]
    ev1.record(stream)
    ev1.synchronize()
    dts_s = ev0.elapsed_time(ev1) / 1000.0
    for r in dts:
        r.close()

    # end to end: plan + launch + every result fetched to the host, per batch
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(args.e2e_steps):
        res = batch_step()
        for r in res:
            d2h = d2h + sum(o.nbytes for o in cq.fetch_all(r))
            r.close()
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    d2h //= args.e2e_steps

    per_step = elapsed / args.steps
    line = {
        "metric": METRIC, "value": rows / per_step, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_step * 1000, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"batched-{args.queries}q-{len(parts)}parts", "queries": args.queries,
                   "partitions": len(parts), "pool_rows": int(sizes.sum()), "logical_rows_per_batch": rows,
                   "compressed_bytes_per_batch": nbytes, "tuned": {"tile_rows": best.tile_rows,
                                                                    "items_per_cta": best.items_per_cta,
                                                                    "launch_us": tuned_us},
                   "pool_generation_s": t_gen, "parallelism": "replicas1",
                   "l2": "each batch reads far more than L2 (129 MB); no flush"},
        "queries_per_s": args.queries / per_step,
        "compressed_gbs": nbytes / per_step / 1e9,
        "pct_hbm_peak": nbytes / per_step / 1e9 / peak,
        "launch_us_median": statistics.median(launch_us),
        "host_submit_ms_per_batch": 1000 * t_host / args.steps,
        "one_query_at_a_time": {"queries_per_s": len(handles) / solo_s, "rows_per_s": rows / solo_s,
                                "speedup_of_batch": solo_s / per_step},
        "decompress_then_scan": {"queries": n_dts, "queries_per_s": n_dts / dts_s, "rows_per_s": dts_rows / dts_s},
        "roofline": {"bound": "hbm", "achieved": nbytes / per_step / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": nbytes / per_step / 1e9 / peak, "traffic": None, "kernel": "batch_query_kernel",
                     "peak_source": f"{peak_src} hbm_gbs", "algorithmic_bytes_per_launch": nbytes},
        "e2e": {"value": rows / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h,
                "note": "tables resident; per batch: plan, launch, fetch every result"},
        "clocks": clk,
        "gpu_launches": 5 * args.steps,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- serving workload
def run_serving(args):
    """Poisson arrivals over resident tables (60% two-RLE 1M-row table, 30%
    heterogeneous 100M-row table, 10% nested partitions), served by the
    continuous-batching loop, by one query at a time, and by one query at a
    time on the decompress-then-scan path; p50 / p99 latency and achieved
    queries/s per arrival rate."""
    import threading
    import numpy as np
    import torch
    from paper_2506_10092_gb300 import cq, devgen
    from paper_2506_10092_gb300 import datagen as dg

    torch.cuda.set_device(0)
    ctx = cq.cq_ctx_create(0)
    tiny_t, _ = dg.tiny_two_rle(1_000_000, seed=args.seed)
    het_t, het_plan = dg.heterogeneous(100_000_000, seed=args.seed)
    tiny = cq.table_from(ctx, tiny_t)
    het = cq.table_from(ctx, het_t)
    del het_t
    rng = np.random.default_rng([args.seed, 6])
    nest = [devgen.DeviceNested(cq, ctx, int(n), seed=args.seed + 3000 + i)
            for i, n in enumerate(dg.partition_sizes(rng, 16, 1e4, args.part_max))]
    torch.cuda.synchronize()

    def request(r):
        u = r.random()
        if u < 0.6:
            return tiny[0], cq.PlanStruct(dg.tiny_plan(int(r.integers(0, 100))))
        if u < 0.9:
            lo = int(r.integers(0, 750_001))
            return het[0], cq.PlanStruct(dg.Plan([het_plan.preds[0], dg.Pred(3, "between", lo, lo + 249_999)],
                                                 het_plan.group_by, het_plan.aggs))
        lo = int(r.integers(0, 1000))
        return nest[int(r.integers(0, len(nest)))].table, cq.PlanStruct(dg.nested_plan(lo, min(999, lo + 499),
                                                                                        lean=True))

    def pct(xs, p):
        return float(np.percentile(np.asarray(xs), p)) if xs else None

    # compile the kernels specialised to every query shape of the mix before
    # any timing (each process compiles a shape once): alone and through a
    # server (whose small lane plans queries for batches)
    warm = ([tiny[0], cq.PlanStruct(dg.tiny_plan(50))], [het[0], cq.PlanStruct(het_plan)]) + tuple(
        [p.table, cq.PlanStruct(dg.nested_plan(200, 699, lean=True))] for p in nest)
    for tb, ps in warm:
        cq.cq_result_wait(cq.cq_query_run(tb, ps))
    srv = cq.cq_server_create(ctx, cq.server_options(max_batch=256, n_streams=4, max_wait_us=200))
    for tk in [cq.cq_server_submit(srv, tb, ps) for tb, ps in warm]:
        cq.cq_server_wait(srv, tk)[0].close()
    srv.close()

    def run_mode(mode, rate, reqs, arrivals, n_warm):
        n = len(reqs)
        lat = [None] * n
        done_t = [0.0] * n
        t0 = time.perf_counter() + 0.05
        if mode == "batched":
            srv = cq.cq_server_create(ctx, cq.server_options(max_batch=256, n_streams=4, max_wait_us=200))
            tickets = [None] * n
            got = threading.Event()

            def submit():
                for i, (tb, ps) in enumerate(reqs):
                    dt = t0 + arrivals[i] - time.perf_counter()
                    if dt > 0:
                        time.sleep(dt)
                    tickets[i] = cq.cq_server_submit(srv, tb, ps)
                    if i == 0:
                        got.set()
            th = threading.Thread(target=submit)
            th.start()
            for i in range(n):
                while tickets[i] is None:
                    time.sleep(5e-5)
                res, us = cq.cq_server_wait(srv, tickets[i])
                lat[i] = us
                done_t[i] = time.perf_counter()
                res.close()
            th.join()
            launches, _ = cq.cq_server_stats(srv)
            srv.close()
        else:
            opts = cq.exec_options(mode=cq.CQ_EXEC_DECOMPRESS_THEN_SCAN) if mode == "decompress_then_scan" else None
            launches = n
            for i, (tb, ps) in enumerate(reqs):
                arr = t0 + arrivals[i]
                dt = arr - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                r = cq.cq_query_run(tb, ps, opts=opts)
                cq.cq_result_wait(r)
                done_t[i] = time.perf_counter()
                lat[i] = (done_t[i] - arr) * 1e6
                r.close()
        # statistics over the measured arrivals only (after the warm-up ones)
        meas = lat[n_warm:]
        t_first = t0 + arrivals[n_warm] if n_warm < n else t0
        span = max(done_t[n_warm:]) - t_first
        return {"mode": mode, "rate": rate, "queries": n - n_warm, "warmup_queries": n_warm,
                "achieved_qps": (n - n_warm) / span, "p50_us": pct(meas, 50), "p99_us": pct(meas, 99),
                "p99_samples": len(meas), "launches": launches}

    rows = []
    modes = [m for m in args.serve_modes.split(",") if m]
    for rate in [float(x) for x in args.rates.split(",")]:
        n_warm = int(rate * args.serve_warmup)
        n = n_warm + max(20, int(rate * args.serve_seconds))
        r = np.random.default_rng([args.seed, 7, int(rate)])
        arrivals = np.cumsum(r.exponential(1.0 / rate, size=n))
        reqs = [request(r) for _ in range(n)]
        for mode in modes:
            # the comparison path is slow: a bounded prefix of the same arrivals
            k = n if mode != "decompress_then_scan" else min(n, n_warm + 1500)
            rows.append(run_mode(mode, rate, reqs[:k], arrivals[:k], min(n_warm, k - 1)))
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    best = max((x for x in rows if x["mode"] == "batched"), key=lambda x: x["achieved_qps"], default=None)
    line = {
        "metric": "served queries/s", "value": best["achieved_qps"] if best else None, "unit": "queries/s",
        "n_gpus": 1, "steps": len(rows), "warmup": 0, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": "serving-mix-60-30-10", "rates": args.rates, "seconds_per_rate": args.serve_seconds,
                   "warmup_seconds_per_rate": args.serve_warmup,
                   "tables": "two-RLE 1M, heterogeneous 100M, 16 nested partitions", "parallelism": "replicas1"},
        "p50_us": best["p50_us"] if best else None, "p99_us": best["p99_us"] if best else None,
        "by_rate": rows,
        "gpu_launches": sum(x["launches"] for x in rows),
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "runsweep":
        run_runsweep(args)
    else:
        run_cq(args)


if __name__ == "__main__":
    main()
