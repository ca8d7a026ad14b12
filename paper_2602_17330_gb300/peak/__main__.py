"""python -m paper_2602_17330_gb300.peak [--json PATH]

Compiles alu_peak.cu for sm_103a, runs it on device 0 and prints lane-operations
per SM per clock for each probed operation; with --json the figures are also
written to PATH as {"device": ..., "sms": ..., "ops": {name: rate}, "command":
..., "date": ...}.
"""
import datetime
import json
import os
import re
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
src = os.path.join(HERE, "alu_peak.cu")
exe = os.path.join(HERE, "alu_peak")
subprocess.check_call(["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src])
res = subprocess.run([exe], capture_output=True, text=True)
sys.stdout.write(res.stdout)
sys.stderr.write(res.stderr)
if res.returncode == 0 and "--json" in sys.argv:
    path = sys.argv[sys.argv.index("--json") + 1]
    ops = {}
    device, sms = None, None
    for line in res.stdout.splitlines():
        m = re.match(r"device (.+), (\d+) SMs", line)
        if m:
            device, sms = m.group(1), int(m.group(2))
            continue
        m = re.match(r"(.+?)\s+([0-9.]+) lane-(ops|loads)/SM/clk", line)
        if m:
            ops[m.group(1).strip()] = float(m.group(2))
    with open(path, "w") as fh:
        json.dump({"device": device, "sms": sms, "unit": "lane-ops per SM per clock (busy clock64 cycles)",
                   "ops": ops, "command": "python -m paper_2602_17330_gb300.peak --json " + path,
                   "date": datetime.datetime.now(datetime.timezone.utc).strftime("%Y-%m-%dT%H:%M:%SZ")}, fh, indent=1)
sys.exit(res.returncode)
