"""Hardware probes.  ``python -m paper_2502_11686_gb300.probes`` compiles fma_probe.cu for
sm_103a next to this file and prints the DFMA / FFMA rates it measures."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def run_fma_probe() -> str:
    from ..build import GENCODE, nvcc
    src = os.path.join(HERE, "fma_probe.cu")
    exe = os.path.join(HERE, "fma_probe")
    subprocess.check_call([nvcc(), "-O3", GENCODE, "-o", exe, src])
    return subprocess.check_output([exe], text=True)


if __name__ == "__main__":
    sys.stdout.write(run_fma_probe())
