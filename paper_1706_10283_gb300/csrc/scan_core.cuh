// Vectorized table lookup for the Bolt scan (Sec. 3.2: lookups of V
// consecutive codes per instruction from a 16-entry table of 8-bit entries,
// codes stored in blocks).  On sm_103a the lookup is the prmt byte permute:
// one prmt reads 4 codes' low 3 bits as selectors into an 8-entry half of
// the table, a second prmt reads the other half, and bit 3 of each code
// picks between them.
//
// Per lane and code word W (8 vectors of one codebook; vector i in bits
// [4i, 4i+4)) the kernel accumulates exact per-vector sums (Sec. 3.1,
// sum_m D[h(x)_m, m]) in two 32-bit registers per 4 vectors:
//   full += r          (r = looked-up bytes of vectors 0..3: mod 2^32)
//   odd  += bytes 1, 3 of r placed in 16-bit lanes
// and recovers even = full - (odd << 8) at the end (exact for sums < 2^16,
// i.e. M <= 257 tables of 8-bit entries).
#pragma once

#include "common.cuh"

namespace bolt {

// Multipliers kept in constant memory so the compiler cannot fold them: the
// adds and the left shift of the lookup then issue as IMAD on the FMA pipe,
// leaving the integer ALU pipe (which runs prmt and lop3) to the lookups.
__constant__ uint32_t kMulOne = 1u;
__constant__ uint32_t kMulShl4 = 16u;
__constant__ uint32_t kMulNeg256 = 0xFFFFFF00u;  // -256 mod 2^32

__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

struct WordSel {
    uint32_t s_lo;  // low 3 code bits of vectors 0..3 as prmt selectors (low 16 bits)
    uint32_t s_hi;  // same for vectors 4..7
    uint32_t m_lo;  // byte i = 0xFF iff code of vector i has bit 3 set (i = 0..3)
    uint32_t m_hi;  // same for vectors 4..7
};

__device__ __forceinline__ WordSel prep_word(uint32_t W) {
    WordSel r;
    const uint32_t s7 = W & 0x77777777u;
    r.s_lo = s7;
    r.s_hi = s7 >> 16;
    const uint32_t Wsh = imad(W, kMulShl4, 0u);  // W << 4
    // Sign-replicating selectors: output byte i copies the top bit of the byte
    // holding bit 3 of vector i's code (bit 3 of W's byte, shifted into bit 7
    // of Wsh's byte for even vectors).
    r.m_lo = prmt(Wsh, W, 0xD9C8u);
    r.m_hi = prmt(Wsh, W, 0xFBEAu);
    return r;
}

// Look up 4 vectors in one 16-byte table (t0..t3 = entries 0..15).
__device__ __forceinline__ uint32_t lookup4(uint32_t t0, uint32_t t1, uint32_t t2, uint32_t t3, uint32_t sel,
                                            uint32_t mask) {
    const uint32_t lo = prmt(t0, t1, sel);
    const uint32_t hi = prmt(t2, t3, sel);
    return (hi & mask) | (lo & ~mask);
}

struct Acc8 {
    uint32_t full_lo, odd_lo, full_hi, odd_hi;
    __device__ __forceinline__ void zero() { full_lo = odd_lo = full_hi = odd_hi = 0u; }
    __device__ __forceinline__ void add(const WordSel &w, uint4 t) {
        const uint32_t ra = lookup4(t.x, t.y, t.z, t.w, w.s_lo, w.m_lo);
        const uint32_t rb = lookup4(t.x, t.y, t.z, t.w, w.s_hi, w.m_hi);
        const uint32_t one = kMulOne;
        full_lo = imad(ra, one, full_lo);
        odd_lo = imad(prmt(ra, 0u, 0x4341u), one, odd_lo);
        full_hi = imad(rb, one, full_hi);
        odd_hi = imad(prmt(rb, 0u, 0x4341u), one, odd_hi);
    }
    // Packed results: e = (S0 | S2 << 16), o = (S1 | S3 << 16) etc.
    __device__ __forceinline__ void finish(uint32_t &e_lo, uint32_t &o_lo, uint32_t &e_hi,
                                           uint32_t &o_hi) const {
        o_lo = odd_lo;
        o_hi = odd_hi;
        // full - (odd << 8), as one multiply-add on the FMA pipe
        e_lo = imad(odd_lo, kMulNeg256, full_lo);
        e_hi = imad(odd_hi, kMulNeg256, full_hi);
    }
};

// The 8 sums of a lane as uint16 in vector order 0..7 (4 words).
__device__ __forceinline__ uint4 pack_sums(uint32_t e_lo, uint32_t o_lo, uint32_t e_hi, uint32_t o_hi) {
    uint4 r;
    r.x = prmt(e_lo, o_lo, 0x5410u);
    r.y = prmt(e_lo, o_lo, 0x7632u);
    r.z = prmt(e_hi, o_hi, 0x5410u);
    r.w = prmt(e_hi, o_hi, 0x7632u);
    return r;
}

}  // namespace bolt
