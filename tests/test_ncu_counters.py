"""The bridge from ncu measurements to ktune_step's counters
(paper_2102_05297_gb300.ncu_counters): the table's metric names in the
library's role order, the ncu command (clocks left alone), the CSV parser on
ncu's per-launch, per-metric layout, and the conversions."""
import os
import re

import numpy as np

import workloads as W
from oracle import expert
from paper_2102_05297_gb300 import ncu_counters as nc

HEADER = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",'
          '"Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit",'
          '"Metric Value"')


def row(launch, kernel, metric, unit, value):
    return ('"%d","832","app","127.0.0.1","%s","1","13","(256, 1, 1)","(1216, 1, 1)","0","10.3",'
            '"Command line profiler metrics","%s","%s","%s"' % (launch, kernel, metric, unit, value))


def test_role_order_matches_library():
    assert nc.ROLE_NAMES == W.ROLE_NAMES
    with open(os.path.join(os.path.dirname(__file__), "..", "include", "ktune.h")) as f:
        text = f.read()
    enum = re.search(r"KTUNE_PC_DRAM_RT = 0,(.*?)KTUNE_PC_N_ROLES", text, re.S).group(0)
    names = re.findall(r"KTUNE_PC_(\w+)", enum)[:-1]
    assert names == nc.ROLE_NAMES


def test_metrics_and_command():
    roles = W.layout(32)
    m = nc.metrics_for(roles)
    assert len(m) == len(set(m)) == 24 + 2           # the table's 24, grid and block size
    assert set(nc.TABLE_METRICS.values()) <= set(m)
    cmd = nc.ncu_command(["./app", "--n", "4"], "coulomb", roles, "out.csv", 2, 3)
    assert cmd[:3] == ["ncu", "--clock-control", "none"]
    assert cmd[-3:] == ["./app", "--n", "4"] and "regex:coulomb" in cmd
    assert nc.metrics_for(W.layout(16)) == [nc.TABLE_METRICS[W.ROLE_NAMES[r]] for r in W.layout(16)]


def test_parse_and_convert():
    vals = {nc.TABLE_METRICS[n]: float(i + 1) * 1000 for i, n in enumerate(nc.TABLE_METRICS)}
    vals[nc.TABLE_METRICS["WARP_E"]] = 24.0          # threads per warp instruction
    vals[nc.TABLE_METRICS["DRAM_U"]] = 63.5
    vals["launch__grid_size"] = 1216
    vals["launch__block_size"] = 256
    lines = ["==PROF== Connected to process 832", HEADER]
    for launch, scale in ((0, 1.0), (1, 2.0)):
        for name, v in vals.items():
            unit = "%" if "pct" in name else ("Kbyte" if name == "dram__sectors_read.sum" else "")
            shown = v * scale / 1000 if unit == "Kbyte" else v * scale
            lines.append(row(launch, "coulomb(float4 *, int)", name, unit, "{:,.4f}".format(shown)))
        lines.append(row(launch, "other(int)", "smsp__inst_executed.sum", "inst", "7"))
    launches = nc.parse_csv("\n".join(lines), kernel="coulomb")
    assert len(launches) == 2
    np.testing.assert_allclose(launches[1]["dram__sectors_read.sum"], 2 * vals["dram__sectors_read.sum"])
    assert len(nc.parse_csv("\n".join(lines))) == 2 and nc.parse_csv("") == []
    roles = W.layout(32)
    c = nc.counters(launches[0], roles)
    by = {W.ROLE_NAMES[r]: c[k] for k, r in enumerate(roles) if W.ROLE_NAMES[r] != "INERT"}
    assert by["WARP_E"] == np.float32(75.0)
    assert by["GLOBAL"] == np.float32(1216 * 256)
    assert by["DRAM_U"] == np.float32(63.5)
    l2 = vals[nc.TABLE_METRICS["L2_RT"]] + vals[nc.TABLE_METRICS["L2_WT"]]
    assert by["LOC_O"] == np.float32(min(100.0, 100.0 * vals[nc.TABLE_METRICS["LOC_O"]] / l2))
    assert np.all(c[[k for k, r in enumerate(roles) if W.ROLE_NAMES[r] == "INERT"]] == 0)
    d = expert.delta_vector(roles, c, 0.7, 1000.0)    # the expert system takes them as they are
    assert np.all(np.isfinite(d)) and np.all(np.abs(d) <= 1)


def test_command_line(tmp_path, capsys):
    import json
    vals = {nc.TABLE_METRICS["DRAM_RT"]: 1234.0, nc.TABLE_METRICS["WARP_E"]: 16.0}
    lines = [HEADER] + [row(0, "k(int)", m, "", v) for m, v in vals.items()]
    f = tmp_path / "p.csv"
    f.write_text("\n".join(lines))
    assert nc.main([str(f), "DRAM_RT,WARP_E,25", "--kernel", "k("]) == 0
    assert json.loads(capsys.readouterr().out) == [1234.0, 50.0, 0.0]
