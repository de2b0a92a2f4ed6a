"""Build and run the ALU instruction-rate microbenchmark (alu_rates.cu) on GPU 0 and print
its JSON: warp instructions per SM per clock for each instruction form the max-norm kernels
use, and the SM clock seen."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
BIN = os.path.join(HERE, "_build", "alu_rates")


def build() -> str:
    os.makedirs(os.path.dirname(BIN), exist_ok=True)
    src = os.path.join(HERE, "alu_rates.cu")
    if not os.path.exists(BIN) or os.path.getmtime(BIN) < os.path.getmtime(src):
        subprocess.run(["nvcc", "-O3", "-gencode", "arch=compute_103a,code=sm_103a", "-o", BIN, src],
                       check=True)
    return BIN


if __name__ == "__main__":
    out = subprocess.run([build()], capture_output=True, text=True)
    sys.stdout.write(out.stdout)
    sys.stderr.write(out.stderr)
    sys.exit(out.returncode)
