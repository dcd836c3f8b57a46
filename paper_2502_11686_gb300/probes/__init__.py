"""Hardware probes, compiled for sm_103a next to this file.

``python -m paper_2502_11686_gb300.probes`` prints the DFMA / FFMA rates fma_probe.cu measures;
``python -m paper_2502_11686_gb300.probes tc`` runs tc_probe.cu, which checks the tcgen05
conventions of the tensor-core kernels (TMEM layouts, descriptors, 3xTF32) against an FP64
product and exits non-zero on a mismatch."""
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


def run_tc_probe() -> int:
    from ..build import GENCODE, INCLUDE, nvcc
    src = os.path.join(HERE, "tc_probe.cu")
    exe = os.path.join(HERE, "tc_probe")
    subprocess.check_call([nvcc(), "-O3", GENCODE, "-I", INCLUDE, "-o", exe, src])
    return subprocess.call([exe])


if __name__ == "__main__":
    sys.stdout.write(run_fma_probe())
