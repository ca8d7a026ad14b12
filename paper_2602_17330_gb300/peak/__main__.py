import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
src = os.path.join(HERE, "alu_peak.cu")
exe = os.path.join(HERE, "alu_peak")
subprocess.check_call(["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src])
sys.exit(subprocess.call([exe]))
