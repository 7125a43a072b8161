"""Build and run fp64_peak.cu (nvcc, sm_103a) and print its table.

  python paper_2001_01570_gb300/peak/measure_fp64_peak.py

The DFMA line, times 2 flops per FMA, is the FP64 peak the benchmark's roofline divides by.
"""
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "fp64_peak")
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                        os.path.join(HERE, "fp64_peak.cu")], check=True)
        r = subprocess.run([exe], capture_output=True, text=True)
        sys.stdout.write(r.stdout)
        sys.stderr.write(r.stderr)
        return r.returncode


if __name__ == "__main__":
    sys.exit(main())
