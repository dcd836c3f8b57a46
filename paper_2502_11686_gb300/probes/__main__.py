import sys

from . import run_fma_probe

sys.stdout.write(run_fma_probe())
