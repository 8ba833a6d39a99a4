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

with the SM count read from the device, the maximum SM clock from
nvidia-smi (clocks.max.sm), and the lane rate measured on the device by
bolt_probe_int_lanes (a loop of independent prmt instructions; 64 lanes per
clock per SM on GB300, the rate at which ncu's ALU-pipe utilization of the
lookup kernels reads 100%).
"""
import subprocess

ALU_OPS_PER_LOOKUP = 1.0  # byte-permute lookup floor, selector preparation amortized
ALU_OPS_PER_LOOKUP_ONE_QUERY = 1.5  # selector preparation paid for every lookup word

_cache = {}


def device_numbers():
    """(SMs, maximum SM clock in Hz, ALU lanes per clock per SM, source text)."""
    if "v" not in _cache:
        import torch

        from . import bolt

        dev = torch.cuda.current_device()
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = None
        try:
            out = subprocess.run(["nvidia-smi", "-i", str(dev), "--query-gpu=clocks.max.sm",
                                  "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
            mhz = float(out.stdout.strip().splitlines()[0])
        except Exception:
            mhz = None
        clock_src = "nvidia-smi clocks.max.sm"
        if not mhz:
            mhz, clock_src = 2070.0, "GB300 maximum SM clock (nvidia-smi unavailable)"
        lanes = bolt.probe_int_lanes()
        src = ("%d SMs x %.1f int32 ALU lanes/clk (bolt_probe_int_lanes) x %.0f MHz (%s) / 1 ALU op per lookup "
               "(byte-permute floor; one-query-per-pass kernels are capped at 2/3 of it)" % (sms, lanes, mhz,
                                                                                            clock_src))
        _cache["v"] = (sms, mhz * 1e6, lanes, src)
    return _cache["v"]


def int_ops_per_s():
    sms, hz, lanes, _ = device_numbers()
    return sms * lanes * hz


def lookups_per_s():
    return int_ops_per_s() / ALU_OPS_PER_LOOKUP


def lookups_per_s_one_query():
    return int_ops_per_s() / ALU_OPS_PER_LOOKUP_ONE_QUERY


def source():
    return device_numbers()[3]
