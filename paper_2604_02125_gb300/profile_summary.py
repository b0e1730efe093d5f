"""Short text summaries of Nsight Compute output for the profiles folder.

Two modes:

  launch list (a `--metrics gpu__time_duration.sum --csv --log-file X.csv` run):
    python -m paper_2604_02125_gb300.profile_summary launches X.csv --out profiles/NAME.md \
        --command "<the ncu command line>"
  per kernel, launch count, total device time and share of the total.

  kernel capture (a `--set full -o X` run; X.ncu-rep, or the output of
  `ncu -i X.ncu-rep --page raw --csv` saved as a .csv):
    python -m paper_2604_02125_gb300.profile_summary kernel X.ncu-rep --kernel REGEX --out profiles/NAME.md \
        --command "<the ncu command line>" --workload "<what ran>"
  duration, DRAM bytes, pipe utilisations, occupancy and stall reasons of
  every captured launch of the kernel, plus two machine-readable lines,
  `dram_bytes_per_launch:` and `source_sha256:` (a hash of the kernel sources,
  see kernel_source_hash), from which bench.py takes the roofline's traffic
  while the kernel sources are unchanged.
"""
import argparse
import csv
import hashlib
import io
import os
import re
import statistics
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")

# sources whose code ends up in the lane-form volume and face kernels
KERNEL_SOURCES = ("crkfr_physics.cuh", "crkfr_f2.cuh", "crkfr_kernels.cuh", "crkfr_async.cuh",
                  "crkfr_volume_lanes.cuh", "cr_variant.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def _num(s):
    try:
        return float(str(s).replace(",", ""))
    except ValueError:
        return None


def summarize_launches(path):
    """{kernel name: (launches, total ns)} from an ncu --csv launch list."""
    with open(path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    rows = list(csv.DictReader(io.StringIO("".join(lines))))
    agg = {}
    for r in rows:
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        ns = _num(r["Metric Value"])
        scale = {"ns": 1.0, "us": 1e3, "usecond": 1e3, "ms": 1e6, "msecond": 1e6, "nsecond": 1.0}.get(
            r.get("Metric Unit", "ns"), 1.0)
        name = re.sub(r"\(.*", "", r["Kernel Name"]).replace("void ", "").strip()
        c, t = agg.get(name, (0, 0.0))
        agg[name] = (c + 1, t + ns * scale)
    return agg


def launches_markdown(path, command):
    agg = summarize_launches(path)
    total = sum(t for _, t in agg.values()) or 1.0
    out = ["# Launch list", "", "Command:", "", "```", command, "```", "",
           "Per-launch times under ncu are cold-cache and serialised: compare shares, not absolutes.", "",
           "| kernel | launches | total us | mean us | share |", "|---|---:|---:|---:|---:|"]
    for name, (c, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        out.append("| `%s` | %d | %.1f | %.2f | %.3f |" % (name, c, t / 1e3, t / 1e3 / c, t / total))
    out.append("")
    return "\n".join(out)


KERNEL_METRICS = [
    ("duration", "gpu__time_duration.sum"),
    ("DRAM read", "dram__bytes_read.sum"),
    ("DRAM write", "dram__bytes_write.sum"),
    ("DRAM throughput % of peak", "gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed"),
    ("L2 sector hit rate (bytes served by L2 are not HBM traffic)", "lts__t_sector_hit_rate.pct"),
    ("L2 read hit rate", "lts__t_sector_op_read_hit_rate.pct"),
    ("L1 sector hit rate", "l1tex__t_sector_hit_rate.pct"),
    ("registers / thread", "launch__registers_per_thread"),
    ("block size", "launch__block_size"),
    ("grid size", "launch__grid_size"),
    ("dynamic shared memory / block", "launch__shared_mem_per_block_dynamic"),
    ("warps active % of peak", "sm__warps_active.avg.pct_of_peak_sustained_active"),
    ("issue active %", "smsp__issue_active.avg.pct_of_peak_sustained_active"),
    ("warp instructions executed", "smsp__inst_executed.sum"),
    ("FMA pipe %", "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active"),
    ("ALU pipe %", "sm__pipe_alu_cycles_active.avg.pct_of_peak_sustained_active"),
    ("FP64 pipe %", "sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active"),
    ("XU (MUFU) pipe %", "sm__pipe_xu_cycles_active.avg.pct_of_peak_sustained_active"),
    ("LSU instructions %", "sm__inst_executed_pipe_lsu.avg.pct_of_peak_sustained_active"),
    ("shared-memory bank conflicts", "l1tex__data_bank_conflicts_pipe_lsu_mem_shared.sum"),
    ("eligible warps / cycle", "smsp__warps_eligible.avg.per_cycle_active"),
]
STALL = re.compile(r"smsp__average_warps_issue_stalled_(\w+)_per_issue_active\.ratio")


def kernel_rows(rep, kernel_regex):
    """Rows of the captured launches of a kernel: from an .ncu-rep (read with
    `ncu -i REP --page raw --csv`) or from that command's saved output (.csv)."""
    if rep.endswith(".csv"):
        with open(rep) as f:
            out = f.read()
    else:
        out = subprocess.run(["ncu", "-i", rep, "--page", "raw", "--csv"], capture_output=True, text=True,
                             check=True).stdout
    rows = list(csv.reader(out.splitlines()))
    head, units = rows[0], rows[1]
    pat = re.compile(kernel_regex)
    found = []
    for r in rows[2:]:
        d = dict(zip(head, r))
        if pat.search(d.get("Kernel Name", "")):
            found.append((d, dict(zip(head, units))))
    return found


def kernel_markdown(rep, kernel_regex, command, workload):
    found = kernel_rows(rep, kernel_regex)
    if not found:
        raise SystemExit("no launch of %r in %s" % (kernel_regex, rep))
    name = found[0][0]["Kernel Name"]
    out = ["# %s" % re.sub(r"\(.*", "", name).replace("void ", ""), "", "Workload: %s" % workload, "",
           "Command:", "", "```", command, "```", "",
           "| metric | " + " | ".join("launch %d" % i for i in range(len(found))) + " | unit |",
           "|---|" + "---:|" * len(found) + "---|"]
    for label, key in KERNEL_METRICS:
        if key in found[0][0]:
            out.append("| %s (`%s`) | " % (label, key) + " | ".join(d[key] for d, _ in found)
                       + " | %s |" % found[0][1].get(key, ""))
    stalls = sorted({m.group(1) for k in found[0][0] for m in [STALL.match(k)] if m})
    out += ["", "Warp stall reasons (warps per issued instruction, first launch):", "",
            "| reason | ratio |", "|---|---:|"]
    for s in stalls:
        v = _num(found[0][0]["smsp__average_warps_issue_stalled_%s_per_issue_active.ratio" % s])
        if v is not None and v >= 0.05:
            out.append("| %s | %.3f |" % (s, v))

    def bytes_of(d, u, key):
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}.get(u.get(key, "byte"), 1)
        return _num(d[key]) * scale

    traffic = statistics.mean(bytes_of(d, u, "dram__bytes_read.sum") + bytes_of(d, u, "dram__bytes_write.sum")
                              for d, u in found)
    out += ["", "Machine-readable (read by bench.py):", "", "```",
            "kernel: %s" % re.sub(r"\(.*", "", name).replace("void ", ""),
            "dram_bytes_per_launch: %d" % round(traffic),
            "source_sha256: %s" % kernel_source_hash(), "```", ""]
    return "\n".join(out)


def read_profile_traffic(path):
    """(kernel, dram bytes per launch) from a kernel summary whose source hash
    matches the current kernel sources, else None."""
    try:
        with open(path) as f:
            text = f.read()
    except OSError:
        return None
    kv = dict(re.findall(r"^(kernel|dram_bytes_per_launch|source_sha256): (.+)$", text, re.M))
    if kv.get("source_sha256") != kernel_source_hash() or "dram_bytes_per_launch" not in kv:
        return None
    return kv.get("kernel"), int(kv["dram_bytes_per_launch"])


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="mode", required=True)
    a1 = sub.add_parser("launches")
    a1.add_argument("csv")
    a2 = sub.add_parser("kernel")
    a2.add_argument("rep")
    a2.add_argument("--kernel", required=True)
    a2.add_argument("--workload", required=True)
    for a in (a1, a2):
        a.add_argument("--out", required=True)
        a.add_argument("--command", required=True)
    a = ap.parse_args(argv)
    text = launches_markdown(a.csv, a.command) if a.mode == "launches" else \
        kernel_markdown(a.rep, a.kernel, a.command, a.workload)
    with open(a.out, "w") as f:
        f.write(text)
    return 0


if __name__ == "__main__":
    sys.exit(main())
