import sys

from . import run_fma_probe, run_tc_probe

if len(sys.argv) > 1 and sys.argv[1] == "tc":
    sys.exit(run_tc_probe())
sys.stdout.write(run_fma_probe())
