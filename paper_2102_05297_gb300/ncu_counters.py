"""Measured counters for ``ktune_step``: the Volta-and-newer metrics of the
paper's counter table (Section 3.4, Table "tab:pcs"), an ``ncu`` command that
collects them for one kernel, and the conversion of ``ncu``'s CSV into the
library's counter layout.

Host tooling, off the search step: it turns a profiling run of a real kernel
into the HOST float[K] that ``ktune_step`` takes, in place of the synthetic
performance function.  The metric names are the table's; the conversions
follow its notes and the library's conventions:

  * utilisations (DRAM_U, L2_U, TEX_U, SHR_U, SM_E, INST_ISSUE_U, WARP_NP_E)
    stay percentages in [0, 100] (the library reads X_U as pct / 100);
  * WARP_E = threads per executed warp instruction x 100 / 32 (a percentage);
  * GLOBAL = threads launched (grid size x block size), the parallelism input
    of Section 3.4.2;
  * LOC_O, a percentage before Volta, has only a sector count after it; it is
    read as the local-memory store sectors over all L2 sectors, in percent,
    capped at 100;
  * counts (sectors, requests, wavefronts, instructions) are taken as they are;
  * an inert role reads 0.
"""
from __future__ import annotations

import csv
import io
import re
from typing import Dict, List, Optional, Sequence

import numpy as np

# role name -> Volta+ metric (Table "tab:pcs"), in the table's order
TABLE_METRICS = {
    "DRAM_RT": "dram__sectors_read.sum",
    "DRAM_WT": "dram__sectors_write.sum",
    "L2_RT": "lts__t_sectors_op_read.sum",
    "L2_WT": "lts__t_sectors_op_write.sum",
    "TEX_RWT": "l1tex__t_requests_pipe_lsu_mem_global_op_ld.sum",
    "LOC_O": "l1tex__t_sectors_pipe_lsu_mem_local_op_st.sum",
    "SHR_LT": "l1tex__data_pipe_lsu_wavefronts_mem_shared_op_ld.sum",
    "SHR_WT": "l1tex__data_pipe_lsu_wavefronts_mem_shared_op_st.sum",
    "INST_F32": "smsp__sass_thread_inst_executed_op_fp32_pred_on.sum",
    "INST_F64": "smsp__sass_thread_inst_executed_op_fp64_pred_on.sum",
    "INST_INT": "smsp__sass_thread_inst_executed_op_integer_pred_on.sum",
    "INST_MISC": "smsp__sass_thread_inst_executed_op_misc_pred_on.sum",
    "INST_LDST": "smsp__sass_thread_inst_executed_op_memory_pred_on.sum",
    "INST_CONT": "smsp__sass_thread_inst_executed_op_control_pred_on.sum",
    "INST_BCONV": "smsp__sass_thread_inst_executed_op_conversion_pred_on.sum",
    "INST_EXE": "smsp__inst_executed.sum",
    "INST_ISSUE_U": "smsp__issue_active.avg.pct_of_peak_sustained_active",
    "DRAM_U": "dram__throughput.avg.pct_of_peak_sustained_elapsed",
    "L2_U": "lts__t_sectors.avg.pct_of_peak_sustained_elapsed",
    "TEX_U": "l1tex__t_requests_pipe_lsu_mem_global_op_ld.avg.pct_of_peak_sustained_active",
    "SHR_U": "l1tex__data_pipe_lsu_wavefronts_mem_shared.avg.pct_of_peak_sustained_elapsed",
    "SM_E": "smsp__cycles_active.avg.pct_of_peak_sustained_elapsed",
    "WARP_E": "smsp__thread_inst_executed_per_inst_executed.ratio",
    "WARP_NP_E": "smsp__thread_inst_executed_per_inst_executed.pct",
}
GLOBAL_METRICS = ("launch__grid_size", "launch__block_size")

# the library's role order (include/ktune.h, enum KTUNE_PC_*)
ROLE_NAMES = list(TABLE_METRICS) + ["GLOBAL", "INERT"]

_PREFIX = {"": 1.0, "K": 1e3, "M": 1e6, "G": 1e9, "T": 1e12}


def metrics_for(roles: Sequence[int]) -> List[str]:
    """The ncu metrics a counter layout (KTUNE_PC_* roles) needs."""
    out: List[str] = []

    def add(m):
        if m not in out:
            out.append(m)

    for r in roles:
        name = ROLE_NAMES[r]
        if name == "GLOBAL":
            for m in GLOBAL_METRICS:
                add(m)
        elif name == "LOC_O":
            add(TABLE_METRICS["LOC_O"])
            add(TABLE_METRICS["L2_RT"])
            add(TABLE_METRICS["L2_WT"])
        elif name != "INERT":
            add(TABLE_METRICS[name])
    return out


def ncu_command(program: Sequence[str], kernel_regex: str, roles: Sequence[int], csv_path: str,
                launch_skip: int = 0, launch_count: int = 1) -> List[str]:
    """An ncu command line that profiles launches of one kernel of `program`
    with the layout's metrics, into a CSV file.  The GPU's clocks are left as
    they are (--clock-control none)."""
    return ["ncu", "--clock-control", "none", "--csv", "--print-units", "base",
            "--metrics", ",".join(metrics_for(roles)), "-k", "regex:" + kernel_regex,
            "-s", str(launch_skip), "-c", str(launch_count), "--log-file", csv_path] + list(program)


def _number(value: str, unit: str) -> float:
    v = float(value.replace(",", ""))
    m = re.match(r"^([KMGT]?)(byte|sector|inst|request|wavefront|cycle|thread|warp|block)?", unit or "")
    if m and m.group(2):
        v *= _PREFIX[m.group(1)]
    return v


def parse_csv(text: str, kernel: Optional[str] = None) -> List[Dict[str, float]]:
    """Metric values per profiled launch from ncu's CSV (one row per launch
    and metric: "ID", ..., "Kernel Name", ..., "Metric Name", "Metric Unit",
    "Metric Value"), in launch order; `kernel` keeps the launches whose name
    contains it.  Lines ncu writes around the table are skipped."""
    lines = [ln for ln in text.splitlines() if ln.startswith('"')]
    rows = list(csv.reader(io.StringIO("\n".join(lines))))
    if not rows:
        return []
    head = rows[0]
    ci = {n: head.index(n) for n in ("ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value")}
    launches: Dict[str, Dict[str, float]] = {}
    for r in rows[1:]:
        if len(r) < len(head) or (kernel and kernel not in r[ci["Kernel Name"]]):
            continue
        launches.setdefault(r[ci["ID"]], {})[r[ci["Metric Name"]]] = _number(
            r[ci["Metric Value"]], r[ci["Metric Unit"]])
    return [launches[k] for k in sorted(launches, key=int)]


def counters(values: Dict[str, float], roles: Sequence[int]) -> np.ndarray:
    """The HOST float[K] ktune_step takes, from one launch's metric values."""
    out = np.zeros(len(roles), dtype=np.float32)
    for k, r in enumerate(roles):
        name = ROLE_NAMES[r]
        if name == "INERT":
            v = 0.0
        elif name == "GLOBAL":
            v = values[GLOBAL_METRICS[0]] * values[GLOBAL_METRICS[1]]
        elif name == "WARP_E":
            v = values[TABLE_METRICS["WARP_E"]] * 100.0 / 32.0
        elif name == "LOC_O":
            l2 = values[TABLE_METRICS["L2_RT"]] + values[TABLE_METRICS["L2_WT"]]
            v = min(100.0, 100.0 * values[TABLE_METRICS["LOC_O"]] / l2) if l2 > 0 else 0.0
        else:
            v = values[TABLE_METRICS[name]]
        out[k] = v
    return out


def main(argv: Optional[Sequence[str]] = None) -> int:
    """python -m paper_2102_05297_gb300.ncu_counters CSV ROLES [--kernel NAME]
    prints one JSON list of counters per profiled launch (ROLES: comma-separated
    KTUNE_PC_* role names or numbers, the model's counter layout)."""
    import argparse
    import json
    ap = argparse.ArgumentParser(description="ncu CSV -> ktune_step counters")
    ap.add_argument("csv")
    ap.add_argument("roles")
    ap.add_argument("--kernel", default=None)
    a = ap.parse_args(argv)
    roles = [int(x) if x.isdigit() else ROLE_NAMES.index(x) for x in a.roles.split(",")]
    with open(a.csv) as f:
        for values in parse_csv(f.read(), a.kernel):
            print(json.dumps([float(v) for v in counters(values, roles)]))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
