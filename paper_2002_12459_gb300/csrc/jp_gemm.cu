// Heavy part: matrix construction and the Boolean matrix product
// (Section 2.2 "Join-Project as Matrix Multiplication"; Algorithm 1,
// "M1 <- R^+ adj matrix, M2 <- S^+ adj matrix, M <- M1 x M2").
//
// M1 (heavy x by heavy y) and M2^T (heavy z by heavy y) are stored as dense
// 0/1 byte matrices, K-major (the heavy y index is contiguous), with the byte
// values 0x00 and 0x38, which are 0.0 and 1.0 in FP8 E4M3.  The product runs
// on the 5th-generation tensor cores as tcgen05.mma.kind::f8f6f4 with FP32
// accumulation in tensor memory: every product term is 0 or 1 and every sum
// is a count of witnesses y, which FP32 holds exactly up to 2^24 (and a sum
// of non-negative terms is never rounded to zero, so the test "M_ac > 0" is
// exact at any size).  The epilogue reads each 128 x 256 accumulator tile
// from tensor memory and stores one bit per entry, M_ac > 0, into a row-major
// bitmap G (heavy x by heavy z); the count matrix never reaches HBM.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "jp_internal.cuh"

namespace jp {
namespace {

constexpr int BM = 128;           // rows of A per tile (heavy x)
constexpr int BN = 256;           // rows of B per tile (heavy z), the wide tile; heavy z are
                                  // padded to a multiple of it, so both tile widths fit
constexpr int BK = 128;           // bytes (= FP8 elements) of K per stage
constexpr int STAGES = 4;
constexpr int GROUP_M = 8;          // row tiles per group of the tile order
constexpr int A_STAGE = BM * BK;  // 16 KB
constexpr int GEMM_THREADS = 192;  // warp 0: TMA, warp 1: MMA + TMEM, warps 2..5: epilogue
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s per bounded wait

// Per tile width TBN (rows of B per tile, 128 or 256): the B stage, the stage
// bytes, the shared memory, the TMEM columns (one FP32 accumulator column per
// output column) and the instruction descriptor of tcgen05.mma kind::f8f6f4:
// D = F32 (bits 4-5 = 1), A = B = E4M3 (bits 7-9, 10-12 = 0), both K-major
// (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
template <int TBN> struct Tile {
    static_assert(TBN == 128 || TBN == 256, "tile width");
    static constexpr int B_STAGE = TBN * BK;
    static constexpr int STAGE_BYTES = A_STAGE + B_STAGE;
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
    static constexpr uint32_t TMEM_COLS = TBN;
    static constexpr uint32_t IDESC = (1u << 4) | (0u << 7) | (0u << 10) |
                                      ((uint32_t)(TBN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false (and the status word gets ST_TIMEOUT) after ns nanoseconds.
__device__ bool mbar_wait_for(uint64_t* bar, uint32_t parity, uint32_t* status,
                              unsigned long long ns) {
    if (mbar_try_wait(bar, parity)) return true;
    unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer() - t0 > ns) {
            atomicOr(status, ST_TIMEOUT);
            return false;
        }
    }
    return true;
}

__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t* status) {
    return mbar_wait_for(bar, parity, status, WAIT_NS);
}

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing
// arrives at; the wait must run out after ns and leave ST_TIMEOUT.
__global__ void wait_selftest_kernel(uint32_t* status, unsigned long long ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait_for(&bar, 0, status, ns);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

// Shared-memory matrix descriptor, K-major with the 128-byte swizzle that the
// TMA loads produce: start address >> 4 (bits 0-13), leading byte offset 1
// (unused by swizzled K-major layouts, bits 16-29), stride byte offset
// 1024 B between 8-row groups (bits 32-45), descriptor version 1 (bits
// 46-47), layout SWIZZLE_128B = 2 (bits 61-63).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// One 128 x TBN output tile per CTA.  K is consumed in BK-byte stages through
// a STAGES-deep TMA ring; each stage feeds BK/32 MMAs (K = 32 per FP8 MMA).
// The epilogue writes one bit per entry (M_ac > 0) into G, or with COUNTS the
// entries themselves (the witness counts, exact below 2^24) as uint32 into G
// read as a count matrix of g_stride entries per row.
template <bool COUNTS, int TBN>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    heavy_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB, int num_kb, uint32_t* __restrict__ G,
                      int64_t g_stride, uint32_t* status, const int2* __restrict__ tiles, int gx,
                      int gy) {
    using T = Tile<TBN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + STAGES * A_STAGE;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * T::STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* accum = empty + STAGES;
    uint64_t* drain = accum + 1;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    // tile order: groups of GROUP_M row tiles, column tiles outer within a group,
    // so that the CTAs resident at one time share a few row blocks of A and
    // column blocks of B that fit in L2 (instead of streaming all of B again
    // for every row block)
    const int gid = blockIdx.x / (GROUP_M * gx);
    const int first_m = gid * GROUP_M;
    const int gsz = min(gy - first_m, GROUP_M);
    const int in_group = blockIdx.x % (GROUP_M * gx);
    const int mi = first_m + in_group % gsz;
    const int nj = in_group / gsz;
    const int m0 = mi * BM;
    const int n0 = nj * TBN;
    // K blocks of this tile: all of them, or (batches) those of the queries its
    // rows and columns share; none shared: the tile's product is zero, written
    // before any barrier or tensor memory is set up
    int kb0 = 0, kb1 = num_kb;
    if (tiles) {
        const int2 t = tiles[(int64_t)mi * gx + nj];
        kb0 = max(t.x, 0);
        kb1 = min(t.y, num_kb);
    }
    if (kb0 >= kb1) {
        if (threadIdx.x >= 64) {               // warps 2-5: one row each thread
            if constexpr (COUNTS) {
                uint4* crow = reinterpret_cast<uint4*>(
                    G + (int64_t)(m0 + (int)threadIdx.x - 64) * g_stride + n0);
                for (int j = 0; j < TBN / 4; ++j) crow[j] = make_uint4(0u, 0u, 0u, 0u);
            } else {
                uint32_t* grow = G + (int64_t)(m0 + (int)threadIdx.x - 64) * g_stride + (n0 >> 5);
#pragma unroll
                for (int j = 0; j < TBN / 32; ++j) grow[j] = 0u;
            }
        }
        return;
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_holder)),
                     "r"(T::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer
        int issued = 0;
        for (int kb = kb0; kb < kb1; ++kb) {
            const int i = kb - kb0;                 // stage and phase count from the first block
            const int s = i % STAGES;
            const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
            if (!mbar_wait(&empty[s], ph ^ 1u, status)) break;
            mbar_arrive_expect_tx(&full[s], T::STAGE_BYTES);
            tma_load_2d(sA + s * A_STAGE, &tmA, &full[s], kb * BK, m0);
            tma_load_2d(sB + s * T::B_STAGE, &tmB, &full[s], kb * BK, n0);
            ++issued;
        }
        // drain: every issued load has landed before the CTA may exit
        for (int i = (issued > STAGES ? issued - STAGES : 0); i < issued; ++i)
            mbar_wait(&full[i % STAGES], (uint32_t)(i / STAGES) & 1u, status);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer (a wait that runs out has set ST_TIMEOUT)
        for (int kb = kb0; kb < kb1; ++kb) {
            const int i = kb - kb0;
            const int s = i % STAGES;
            const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
            if (!mbar_wait(&full[s], ph, status)) break;
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA + s * A_STAGE);
            const uint32_t b0 = smem_u32(sB + s * T::B_STAGE);
#pragma unroll
            for (int k = 0; k < BK / 32; ++k) {
                mma_f8(tmem, sdesc_sw128(a0 + 32 * k), sdesc_sw128(b0 + 32 * k), T::IDESC,
                       (i | k) != 0 ? 1u : 0u);
            }
            mma_commit(&empty[s]);
        }
        mma_commit(accum);
        // wait for every issued MMA before teardown (bounded)
        mma_commit(drain);
        mbar_wait(drain, 0, status);
    } else if (warp >= 2) {
        // ---------------- epilogue: TMEM -> bits -> G
        const int q = warp & 3;                // TMEM lane quadrant of this warp
        const int row = m0 + q * 32 + lane;
        if (mbar_wait(accum, 0, status)) {
            tc_fence_after();
            if constexpr (COUNTS) {
                uint4* crow = reinterpret_cast<uint4*>(G + (int64_t)row * g_stride + n0);
#pragma unroll 1
                for (int j = 0; j < TBN / 32; ++j) {
                    uint32_t r[32];
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(j * 32), r);
#pragma unroll
                    for (int i = 0; i < 32; i += 4)
                        crow[j * 8 + i / 4] = make_uint4(
                            (uint32_t)__uint_as_float(r[i]), (uint32_t)__uint_as_float(r[i + 1]),
                            (uint32_t)__uint_as_float(r[i + 2]), (uint32_t)__uint_as_float(r[i + 3]));
                }
            } else {
                uint32_t* grow = G + (int64_t)row * g_stride + (n0 >> 5);
#pragma unroll 1
                for (int j = 0; j < TBN / 32; ++j) {
                    uint32_t r[32];
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(j * 32), r);
                    uint32_t bits = 0;
#pragma unroll
                    for (int i = 0; i < 32; ++i) bits |= (r[i] != 0u ? 1u : 0u) << i;
                    grow[j] = bits;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(T::TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------- matrix build
__global__ void pack_rows_kernel(const int32_t* row_inv, int64_t nrows, const int32_t* off,
                                 const int32_t* col, const int32_t* col_map, uint8_t* M,
                                 int64_t ld) {
    // block per heavy row: hub rows hold up to ~1e5 entries
    for (int64_t h = blockIdx.x; h < nrows; h += gridDim.x) {
        int32_t a = row_inv[h];
        for (int32_t e = off[a] + threadIdx.x; e < off[a + 1]; e += blockDim.x) {
            int32_t j = col_map[col[e]];
            if (j >= 0) M[h * ld + j] = 0x38;
        }
    }
}

// M2^T: for heavy y column j, every heavy z in S[y] sets B[hz][j]
__global__ void pack_cols_kernel(const int32_t* col_inv, int64_t ncols, const int32_t* off,
                                 const int32_t* rows, const int32_t* row_map, uint8_t* M,
                                 int64_t ld) {
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = warp; j < ncols; j += nwarps) {
        int32_t b = col_inv[j];
        for (int32_t e = off[b] + lane; e < off[b + 1]; e += 32) {
            int32_t l = row_map[rows[e]];
            if (l >= 0) M[(int64_t)l * ld + j] = 0x38;
        }
    }
}

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

PFN_cuTensorMapEncodeTiled_v12000 lookup_encode_fn() {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    JP_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                  cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p)
        throw Error{JP_ECUDA, "cuTensorMapEncodeTiled is not available"};
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
}

// The driver's tensor-map encoder, looked up once (a function-local static is
// initialised by one thread while the others wait; a failed lookup is retried
// by the next call).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = lookup_encode_fn();
    return fn;
}

CUtensorMap make_map(const uint8_t* base, int64_t rows, int64_t k_bytes, int box_rows) {
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)k_bytes, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)k_bytes};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void*)base, dims, strides, box,
                             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error{JP_ECUDA, "cuTensorMapEncodeTiled failed"};
    return m;
}

}  // namespace

namespace {

// ---------------------------------------------------------------- peak rates
// Dense FP8 tcgen05 rate: each CTA issues `iters` rounds of four 128x256x32
// kind::f8f6f4 MMAs (the product kernel's shape) on operands held in shared
// memory, with no loads, into one TMEM accumulator.
__global__ void __launch_bounds__(64, 1) fp8_peak_kernel(int iters, uint32_t* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    using T = Tile<BN>;
    uint8_t* sB = smem + A_STAGE;
    uint64_t* done = reinterpret_cast<uint64_t*>(smem + A_STAGE + T::B_STAGE);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < (A_STAGE + T::B_STAGE) / 16; i += blockDim.x)
        reinterpret_cast<int4*>(smem)[i] = make_int4(0, 0, 0, 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // operands seen by the MMA unit
    if (threadIdx.x == 0) {
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_holder)),
                     "r"(T::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;
    if (warp == 1 && lane == 0) {
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < BK / 32; ++k)
                mma_f8(tmem, sdesc_sw128(a0 + 32 * k), sdesc_sw128(b0 + 32 * k), T::IDESC,
                       (it | k) != 0 ? 1u : 0u);
        }
        mma_commit(done);
        mbar_wait(done, 0, status);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(T::TMEM_COLS)
                     : "memory");
    }
}

// Legacy INT8 tensor rate: every warp issues `iters` rounds of eight
// independent mma.sync m16n8k32 s8 x s8 -> s32.
__global__ void int8_mma_peak_kernel(int iters, int32_t* sink) {
    uint32_t a0 = threadIdx.x, a1 = a0 * 3u, a2 = a0 * 5u, a3 = a0 * 7u, b0 = a0 ^ 0x55u,
             b1 = a0 ^ 0xAAu;
    int32_t c[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                "{%8,%9}, {%0,%1,%2,%3};"
                : "+r"(c[j][0]), "+r"(c[j][1]), "+r"(c[j][2]), "+r"(c[j][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
    int32_t t = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) t += c[j][0] ^ c[j][1] ^ c[j][2] ^ c[j][3];
    if (t == 0x5eed1234) sink[0] = t;                // keeps the loop
}

// last q with begin[q] <= id
__device__ __forceinline__ int32_t query_of(const int32_t* begin, int32_t nq, int32_t id) {
    int32_t lo = 0, hi = nq;
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (begin[mid] <= id) lo = mid; else hi = mid;
    }
    return lo;
}

// first i in [0, n) with ids[i] >= v (ids ascending), n if none
__device__ __forceinline__ int32_t lower_id(const int32_t* ids, int32_t n, int32_t v) {
    int32_t lo = 0, hi = n;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (ids[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Heavy x (rows), heavy z (columns) and heavy y (K) are numbered in id order,
// and ids are in query order, so a tile's rows belong to queries [qm0, qm1],
// its columns to [qn0, qn1], and the queries they share own one contiguous
// range of heavy y.
__global__ void tile_range_kernel(const int32_t* __restrict__ hx_inv, int64_t u,
                                  const int32_t* __restrict__ hz_inv, int64_t w,
                                  const int32_t* __restrict__ hy_inv, int64_t v,
                                  const int32_t* __restrict__ xq_begin,
                                  const int32_t* __restrict__ yq_begin, int32_t nq, int gx,
                                  int gy, int tbn, int2* __restrict__ tiles) {
    const int64_t nt = (int64_t)gx * gy;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t mi = t / gx, nj = t % gx;
        const int64_t r0 = mi * BM, c0 = nj * tbn;
        int2 out = make_int2(0, 0);
        if (r0 < u && c0 < w) {
            const int64_t r1 = min(u, r0 + BM) - 1, c1 = min(w, c0 + tbn) - 1;
            const int32_t qa = max(query_of(xq_begin, nq, hx_inv[r0]), query_of(xq_begin, nq, hz_inv[c0]));
            const int32_t qb = min(query_of(xq_begin, nq, hx_inv[r1]), query_of(xq_begin, nq, hz_inv[c1]));
            if (qa <= qb) {
                const int32_t k0 = lower_id(hy_inv, (int32_t)v, yq_begin[qa]);
                const int32_t k1 = lower_id(hy_inv, (int32_t)v, yq_begin[qb + 1]);
                if (k0 < k1) out = make_int2(k0 / BK, (k1 + BK - 1) / BK);
            }
        }
        tiles[t] = out;
    }
}

}  // namespace

void measure_peaks(int sms, double* fp8_tflops, double* int8_tflops, uint32_t* d_status,
                   Arena& ws, cudaStream_t st) {
    const size_t smem = (size_t)A_STAGE + Tile<BN>::B_STAGE + 1024 + 64;
    smem_limit((const void*)fp8_peak_kernel, smem);
    cudaEvent_t e0, e1;
    JP_CUDA_TRY(cudaEventCreate(&e0));
    JP_CUDA_TRY(cudaEventCreate(&e1));
    float ms = 0;
    // FP8: one CTA per SM, 20000 rounds of 4 MMAs (~ 40 ms at the nominal rate)
    const int iters8 = 20000;
    fp8_peak_kernel<<<sms, 64, smem, st>>>(64, d_status);       // warm-up
    JP_CHECK_LAUNCH();
    JP_CUDA_TRY(cudaEventRecord(e0, st));
    fp8_peak_kernel<<<sms, 64, smem, st>>>(iters8, d_status);
    JP_CHECK_LAUNCH();
    JP_CUDA_TRY(cudaEventRecord(e1, st));
    JP_CUDA_TRY(cudaEventSynchronize(e1));
    JP_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    *fp8_tflops = 2.0 * BM * BN * 32.0 * (BK / 32) * (double)iters8 * sms / (ms * 1e-3) / 1e12;
    // INT8 mma.sync: 8 warps per block, 4 blocks per SM
    int32_t* sink = ws.get<int32_t>(1);
    const int iters = 4096, blocks = sms * 4, threads = 256;
    int8_mma_peak_kernel<<<blocks, threads, 0, st>>>(16, sink);  // warm-up
    JP_CHECK_LAUNCH();
    JP_CUDA_TRY(cudaEventRecord(e0, st));
    int8_mma_peak_kernel<<<blocks, threads, 0, st>>>(iters, sink);
    JP_CHECK_LAUNCH();
    JP_CUDA_TRY(cudaEventRecord(e1, st));
    JP_CUDA_TRY(cudaEventSynchronize(e1));
    JP_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    *int8_tflops = 2.0 * 16 * 8 * 32 * 8.0 * iters * ((double)blocks * threads / 32) / (ms * 1e-3) / 1e12;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

int2* batch_tile_ranges(const Partition& p, const Heavy& h, const int32_t* xq_begin,
                        const int32_t* yq_begin, int32_t nq, Arena& ws, cudaStream_t st) {
    if (!h.present) return nullptr;
    const int gx = (int)(h.w_pad / h.tbn), gy = (int)(h.u_pad / BM);
    int2* tiles = ws.get<int2>((size_t)gx * gy);
    tile_range_kernel<<<grid_for((int64_t)gx * gy, 256, 152 * 4), 256, 0, st>>>(
        p.hx_inv, p.u, p.hz_inv, p.w, p.hy_inv, p.v, xq_begin, yq_begin, nq, gx, gy, h.tbn, tiles);
    JP_CHECK_LAUNCH();
    return tiles;
}

void wait_selftest(uint32_t* d_status, int64_t ns, cudaStream_t st) {
    wait_selftest_kernel<<<1, 32, 0, st>>>(d_status, (unsigned long long)ns);
    JP_CHECK_LAUNCH();
}

void heavy_pack(const Graph& g, const Partition& p, Heavy& h, Arena& ws, cudaStream_t st) {
    h.present = (p.u > 0 && p.v > 0 && p.w > 0);
    if (!h.present) return;
    h.u_pad = round_up(p.u, BM);
    h.w_pad = round_up(p.w, BN);
    h.v_pad = round_up(p.v, BK);
    h.g_stride = h.w_pad / 32;
    h.tbn = BN;
    h.A = reinterpret_cast<uint8_t*>(ws.carve((size_t)(h.u_pad * h.v_pad)));
    h.B = reinterpret_cast<uint8_t*>(ws.carve((size_t)(h.w_pad * h.v_pad)));
    h.G = ws.get<uint32_t>((size_t)(h.u_pad * h.g_stride));
    JP_CUDA_TRY(cudaMemsetAsync(h.A, 0, (size_t)(h.u_pad * h.v_pad), st));
    JP_CUDA_TRY(cudaMemsetAsync(h.B, 0, (size_t)(h.w_pad * h.v_pad), st));
    pack_rows_kernel<<<grid_for(p.u, 1, 152 * 16), 256, 0, st>>>(
        p.hx_inv, p.u, g.rxoff, g.rycol, p.hy, h.A, h.v_pad);
    JP_CHECK_LAUNCH();
    pack_cols_kernel<<<grid_for(p.v * 32, 256, 152 * 16), 256, 0, st>>>(
        p.hy_inv, p.v, g.syoff, g.szcol, p.hz, h.B, h.v_pad);
    JP_CHECK_LAUNCH();
}

int pick_tile(const Heavy& h, int width, int64_t auto_max_tiles) {
    if (width == 128 || width == 256) return width;
    // auto: products with few wide tiles leave SMs idle; narrow tiles double
    // the CTAs (the crossover is measured by the tile autotuner)
    const int64_t wide_tiles = (h.w_pad / BN) * (h.u_pad / BM);
    return wide_tiles <= auto_max_tiles ? 128 : 256;
}

namespace {
template <int TBN>
void launch_gemm(Heavy& h, uint32_t* d_status, cudaStream_t st, const int2* tiles) {
    using T = Tile<TBN>;
    CUtensorMap ma = make_map(h.A, h.u_pad, h.v_pad, BM);
    CUtensorMap mb = make_map(h.B, h.w_pad, h.v_pad, TBN);
    smem_limit((const void*)heavy_gemm_kernel<false, TBN>, T::SMEM);
    const int gx = (int)(h.w_pad / TBN), gy = (int)(h.u_pad / BM);
    heavy_gemm_kernel<false, TBN><<<(unsigned)gx * (unsigned)gy, GEMM_THREADS, T::SMEM, st>>>(
        ma, mb, (int)(h.v_pad / BK), h.G, h.g_stride, d_status, tiles, gx, gy);
    JP_CHECK_LAUNCH();
}
}  // namespace

void heavy_gemm(Heavy& h, const Partition& p, uint32_t* d_status, cudaStream_t st,
                const int2* tiles) {
    (void)p;
    if (!h.present) return;
    tbegin(TM_GEMM);
    if (h.tbn == 128) launch_gemm<128>(h, d_status, st, tiles);
    else launch_gemm<BN>(h, d_status, st, tiles);
    tend(TM_GEMM);
}

void heavy_gemm_counts(const Heavy& h, uint32_t* C, uint32_t* d_status, cudaStream_t st) {
    if (!h.present) return;
    CUtensorMap ma = make_map(h.A, h.u_pad, h.v_pad, BM);
    CUtensorMap mb = make_map(h.B, h.w_pad, h.v_pad, BN);
    smem_limit((const void*)heavy_gemm_kernel<true, BN>, Tile<BN>::SMEM);
    const int gx = (int)(h.w_pad / BN), gy = (int)(h.u_pad / BM);
    tbegin(TM_GEMM);
    heavy_gemm_kernel<true, BN><<<(unsigned)gx * (unsigned)gy, GEMM_THREADS, Tile<BN>::SMEM, st>>>(
        ma, mb, (int)(h.v_pad / BK), C, h.w_pad, d_status, nullptr, gx, gy);
    JP_CHECK_LAUNCH();
    tend(TM_GEMM);
}

}  // namespace jp
