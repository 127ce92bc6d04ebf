// Tensor memory (TMEM) of sm_100-family SMs used as a per-lane scratchpad.
//
// TMEM is 512 columns x 128 lanes of 32-bit cells per SM, allocated per CTA
// in columns (a power of two, at least 32) and written / read with
// tcgen05.st / tcgen05.ld.  Warp w of a CTA reaches the lanes
// [32 (w % 4), 32 (w % 4) + 32): lane i of the warp owns TMEM lane
// 32 (w % 4) + i, so with the 32x32b shape every thread keeps its own row of
// 32-bit cells there, next to (not in) its registers and shared memory.  No
// tensor-core instruction is involved.  Addresses: bits 31..16 lane, 15..0
// column.  All of these are warp-collective (.sync.aligned): every lane of the
// warp executes them together.
#pragma once

#include <cstdint>

namespace dwtfuse {

// Allocates `ncols` columns for this CTA and writes their base address to
// shared memory at *dst; then gives up the CTA's right to allocate again.
// One whole warp calls it.  Blocks until the columns are free (CTAs resident
// on the SM release theirs when they finish).
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(a), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}

// Frees the CTA's columns; the warp that allocated them calls it, after every
// warp's last access (tmem_fence_before + barrier + tmem_fence_after).
__device__ __forceinline__ void tmem_dealloc(uint32_t base, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(base), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// This thread's earlier tcgen05.st have completed (before it reads the cells back).
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// tm_st_xN: r[0..N) into N consecutive columns of this thread's lane.
__device__ __forceinline__ void tm_st_x1(uint32_t ta, const uint32_t *r) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};\n"
                 :
                 : "r"(ta), "r"(r[0])
                 : "memory");
}

__device__ __forceinline__ void tm_st_x2(uint32_t ta, const uint32_t *r) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};\n"
                 :
                 : "r"(ta), "r"(r[0]), "r"(r[1])
                 : "memory");
}

__device__ __forceinline__ void tm_st_x4(uint32_t ta, const uint32_t *r) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};\n"
                 :
                 : "r"(ta), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3])
                 : "memory");
}

__device__ __forceinline__ void tm_st_x8(uint32_t ta, const uint32_t *r) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n"
                 :
                 : "r"(ta), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

__device__ __forceinline__ void tm_st_x16(uint32_t ta, const uint32_t *r) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};\n"
                 :
                 : "r"(ta), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
                 : "memory");
}

__device__ __forceinline__ void tm_st_x32(uint32_t ta, const uint32_t *r) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};\n"
                 :
                 : "r"(ta), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
                 : "memory");
}


// tm_ldnw_xN: N consecutive columns of this thread's lane into r[0..N),
// issued without waiting (tm_wait_ld waits once for all issued loads).
__device__ __forceinline__ void tm_ldnw_x1(uint32_t ta, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];\n" : "=r"(r[0]) : "r"(ta) : "memory");
}

__device__ __forceinline__ void tm_ldnw_x2(uint32_t ta, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(ta) : "memory");
}

__device__ __forceinline__ void tm_ldnw_x4(uint32_t ta, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n" : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(ta) : "memory");
}

__device__ __forceinline__ void tm_ldnw_x8(uint32_t ta, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n" : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]) : "r"(ta) : "memory");
}

__device__ __forceinline__ void tm_ldnw_x16(uint32_t ta, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n" : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]) : "r"(ta) : "memory");
}

__device__ __forceinline__ void tm_ldnw_x32(uint32_t ta, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n" : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]) : "r"(ta) : "memory");
}

// Issues the loads of N columns (power-of-two pieces, N known at compile time).
template <int N>
__device__ __forceinline__ void tm_issue(uint32_t ta, uint32_t *r) {
    if constexpr (N >= 32) {
        tm_ldnw_x32(ta, r);
        tm_issue<N - 32>(ta + 32, r + 32);
    } else if constexpr (N >= 16) {
        tm_ldnw_x16(ta, r);
        tm_issue<N - 16>(ta + 16, r + 16);
    } else if constexpr (N >= 8) {
        tm_ldnw_x8(ta, r);
        tm_issue<N - 8>(ta + 8, r + 8);
    } else if constexpr (N >= 4) {
        tm_ldnw_x4(ta, r);
        tm_issue<N - 4>(ta + 4, r + 4);
    } else if constexpr (N >= 2) {
        tm_ldnw_x2(ta, r);
        tm_issue<N - 2>(ta + 2, r + 2);
    } else if constexpr (N == 1) {
        tm_ldnw_x1(ta, r);
    }
}

// Ties registers to the wait before them: an empty statement that "changes"
// them, so no use of a loaded value is scheduled above the wait.
template <int N>
__device__ __forceinline__ void tm_pin(uint32_t *r) {
    if constexpr (N >= 4) {
        asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]));
        tm_pin<N - 4>(r + 4);
    } else if constexpr (N >= 1) {
        asm volatile("" : "+r"(r[0]));
        tm_pin<N - 1>(r + 1);
    }
}

// Waits for this thread's issued loads; r[0..N) may be used after it.
template <int N>
__device__ __forceinline__ void tm_wait_ld(uint32_t *r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    tm_pin<N>(r);
}

template <int N>
__device__ __forceinline__ void tm_store(uint32_t ta, const uint32_t *r) {
    if constexpr (N >= 32) {
        tm_st_x32(ta, r);
        tm_store<N - 32>(ta + 32, r + 32);
    } else if constexpr (N >= 16) {
        tm_st_x16(ta, r);
        tm_store<N - 16>(ta + 16, r + 16);
    } else if constexpr (N >= 8) {
        tm_st_x8(ta, r);
        tm_store<N - 8>(ta + 8, r + 8);
    } else if constexpr (N >= 4) {
        tm_st_x4(ta, r);
        tm_store<N - 4>(ta + 4, r + 4);
    } else if constexpr (N >= 2) {
        tm_st_x2(ta, r);
        tm_store<N - 2>(ta + 2, r + 2);
    } else if constexpr (N == 1) {
        tm_st_x1(ta, r);
    }
}

}  // namespace dwtfuse
