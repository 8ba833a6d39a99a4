"""Integer-pipe peak used as the roofline of the scan when its codes are
cache resident (or shared by many queries).

The scan's work is one table lookup and one add per (query, vector,
codebook) (Sec. 3.1: Theta(M) per approximate distance).  The byte-permute
lookup does that work four bytes at a time: per 32-bit code word (8
vectors) and query it issues 8 instructions on the integer ALU pipe
(2 x 2 prmt table reads, 2 lop3 half selects, 2 prmt odd-byte splits); the
adds run as imad on the FMA pipe, which issues in parallel.  Preparing a
word's selectors takes 4 more ALU instructions, paid once per word and
shared by every query that scans it.  So the floor is 1 ALU instruction per
lookup (1.5 for a kernel that scans one query per pass), and the peak is

    SMs x ALU lanes per SM per clock x maximum SM clock / 1

with the lane count measured on a GB300 by a throughput loop of independent
prmt / lop3 instructions (INT_LANES_PER_SM).
"""
SMS = 152
MAX_SM_CLOCK_HZ = 2.070e9
INT_LANES_PER_SM = 64  # measured prmt / lop3 throughput per SM per clock
ALU_OPS_PER_LOOKUP = 1.0  # byte-permute lookup floor, selector preparation amortized
ALU_OPS_PER_LOOKUP_ONE_QUERY = 1.5  # selector preparation paid for every lookup word
SOURCE = ("152 SMs x %d int32 ALU lanes/clk x 2070 MHz / 1 ALU op per lookup (byte-permute floor; "
          "one-query-per-pass kernels are capped at 2/3 of it)" % INT_LANES_PER_SM)


def int_ops_per_s():
    return SMS * INT_LANES_PER_SM * MAX_SM_CLOCK_HZ


def lookups_per_s():
    return int_ops_per_s() / ALU_OPS_PER_LOOKUP


def lookups_per_s_one_query():
    return int_ops_per_s() / ALU_OPS_PER_LOOKUP_ONE_QUERY
