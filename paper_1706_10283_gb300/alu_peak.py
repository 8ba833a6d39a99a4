"""Integer-pipe peak used as the roofline of the scan when its codes are
cache resident.

The scan's algorithmic work is one table lookup and one add per (query,
vector, codebook) (Sec. 3.1: Theta(M) per approximate distance), i.e. two
integer operations.  The peak is the GPU's 32-bit integer issue rate,
SMs x integer lanes per SM per clock x maximum SM clock, with the lane count
measured on a GB300 by a throughput loop of independent prmt / lop3 / add
instructions (INT_LANES_PER_SM).
"""
SMS = 152
MAX_SM_CLOCK_HZ = 2.070e9
INT_LANES_PER_SM = 64  # measured: see the integer-throughput note in the design doc
OPS_PER_LOOKUP = 2  # one lookup + one add
SOURCE = "152 SMs x %d int32 lanes/clk x 2070 MHz; 2 ops per lookup-add" % INT_LANES_PER_SM


def int_ops_per_s():
    return SMS * INT_LANES_PER_SM * MAX_SM_CLOCK_HZ


def lookups_per_s():
    return int_ops_per_s() / OPS_PER_LOOKUP
