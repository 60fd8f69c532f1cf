// Cost-filtered nearest neighbour (Alg. 2 NEAREST), radius query (Alg. 2
// NEIGHBORS) and path cost (Sec. III-A) over SoA state-cost trees.
//
// NEAREST, small batches: a block owns QB queries (staged in shared memory)
// and a slice of the tree.  Each thread streams vertices of the slice through
// registers (coalesced SoA rows), evaluates all QB queries against the vertex
// with float4 broadcast reads of the queries, and keeps a running best per
// query under the key (d^2, g, index).  A warp-shuffle argmin and a
// cross-warp pass finish the block; when the tree is split across blocks (few
// queries, large tree), partial bests go to stream-ordered scratch and a
// second kernel reduces them.  Large batches take the budget-ordered path
// further down, whose filter runs on the tensor cores.
#include <algorithm>
#include <cfloat>
#include <cuda_fp16.h>
#include <mutex>

#include "mrpop_internal.cuh"

namespace mrpop {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kNNThreads = 256;
constexpr int kQB = 8;

struct Best {
    float d2;
    float g;
    int idx;
};

// Lexicographic (d^2, g, index); idx < 0 marks "none" (d2 = +inf).
__device__ __forceinline__ bool better(const Best &a, const Best &b) {
    if (a.d2 != b.d2) return a.d2 < b.d2;
    if (a.g != b.g) return a.g < b.g;
    return (unsigned)a.idx < (unsigned)b.idx;
}

__device__ __forceinline__ Best shfl_best(const Best &b, int off) {
    Best o;
    o.d2 = __shfl_xor_sync(kFull, b.d2, off);
    o.g = __shfl_xor_sync(kFull, b.g, off);
    o.idx = __shfl_xor_sync(kFull, b.idx, off);
    return o;
}

template <int DP>
__global__ void __launch_bounds__(kNNThreads)
nearest_kernel(const float *__restrict__ tree, int N, int64_t ld, int dim,
               const float *__restrict__ queries, const float *__restrict__ budgets, int Q,
               int chunk, int64_t *__restrict__ out_idx, Best *__restrict__ partial) {
    __shared__ __align__(16) float qs[kQB][DP];
    __shared__ float cs[kQB];
    __shared__ Best wbest[kNNThreads / 32][kQB];
    const int q0 = blockIdx.x * kQB;
    const int nq = min(kQB, Q - q0);
    for (int i = threadIdx.x; i < kQB * DP; i += blockDim.x) {
        const int j = i / DP, d = i % DP;
        qs[j][d] = (j < nq && d < dim) ? queries[(size_t)d * Q + q0 + j] : 0.f;
    }
    if (threadIdx.x < kQB) cs[threadIdx.x] = threadIdx.x < nq ? budgets[q0 + threadIdx.x] : -FLT_MAX;
    __syncthreads();

    Best best[kQB];
#pragma unroll
    for (int j = 0; j < kQB; ++j) best[j] = Best{FLT_MAX * 2.f, FLT_MAX * 2.f, -1};

    const int vs = blockIdx.y * chunk;
    const int ve = min(N, vs + chunk);
    for (int v = vs + threadIdx.x; v < ve; v += blockDim.x) {
        float x[DP];
#pragma unroll
        for (int d = 0; d < DP; ++d) x[d] = d < dim ? __ldg(tree + (size_t)d * ld + v) : 0.f;
        const float g = __ldg(tree + (size_t)dim * ld + v);
#pragma unroll
        for (int j = 0; j < kQB; ++j) {
            const float4 *q4 = reinterpret_cast<const float4 *>(qs[j]);
            float d2 = 0.f;
#pragma unroll
            for (int d = 0; d < DP / 4; ++d) {
                const float4 qq = q4[d];
                const float a0 = qq.x - x[4 * d], a1 = qq.y - x[4 * d + 1];
                const float a2 = qq.z - x[4 * d + 2], a3 = qq.w - x[4 * d + 3];
                d2 = fmaf(a0, a0, d2);
                d2 = fmaf(a1, a1, d2);
                d2 = fmaf(a2, a2, d2);
                d2 = fmaf(a3, a3, d2);
            }
            if (d2 <= best[j].d2) {
                // filter of Alg. 2: g_v + |q - q_v| < c (strict)
                if (g + __fsqrt_rn(d2) < cs[j] && (d2 < best[j].d2 || g < best[j].g)) {
                    best[j].d2 = d2;
                    best[j].g = g;
                    best[j].idx = v;
                }
            }
        }
    }

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kQB; ++j) {
        Best b = best[j];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const Best o = shfl_best(b, off);
            if (better(o, b)) b = o;
        }
        if (lane == 0) wbest[warp][j] = b;
    }
    __syncthreads();
    if (threadIdx.x < nq) {
        const int j = threadIdx.x;
        Best b = wbest[0][j];
        for (int w = 1; w < kNNThreads / 32; ++w)
            if (better(wbest[w][j], b)) b = wbest[w][j];
        if (partial)
            partial[(size_t)blockIdx.y * Q + q0 + j] = b;
        else
            out_idx[q0 + j] = b.idx;
    }
}

__global__ void nearest_reduce_kernel(const Best *__restrict__ partial, int splits, int Q,
                                      int64_t *__restrict__ out_idx) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    Best b = partial[q];
    for (int s = 1; s < splits; ++s) {
        const Best o = partial[(size_t)s * Q + q];
        if (better(o, b)) b = o;
    }
    out_idx[q] = b.idx;
}

template <int DP>
mrpop_status nearest_dp(const float *tree, int N, int64_t ld, int dim, const float *queries,
                        const float *budgets, int Q, int64_t *out_idx, cudaStream_t st) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int groups = (Q + kQB - 1) / kQB;
    const int target = sms * 8;
    int splits = 1;
    if (groups < target && N > 4 * kNNThreads) {
        splits = (target + groups - 1) / groups;
        splits = std::min(splits, (N + 4 * kNNThreads - 1) / (4 * kNNThreads));
        splits = std::max(splits, 1);
        splits = std::min(splits, 65535);
    }
    int chunk = (N + splits - 1) / splits;
    chunk = ((chunk + kNNThreads - 1) / kNNThreads) * kNNThreads;
    if (chunk == 0) chunk = kNNThreads;
    splits = std::max(1, (N + chunk - 1) / chunk);
    Best *partial = nullptr;
    if (splits > 1)
        MRPOP_CUDA_TRY(scratch_alloc((void **)&partial, sizeof(Best) * (size_t)splits * Q, st));
    dim3 grid(groups, splits);
    nearest_kernel<DP><<<grid, kNNThreads, 0, st>>>(tree, N, ld, dim, queries, budgets, Q, chunk,
                                                    out_idx, partial);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && splits > 1) {
        nearest_reduce_kernel<<<(Q + 255) / 256, 256, 0, st>>>(partial, splits, Q, out_idx);
        e = cudaGetLastError();
    }
    if (partial) cudaFreeAsync(partial, st);
    if (e != cudaSuccess) return cuda_error(e, "nearest kernel launch");
    return MRPOP_OK;
}

// ---------------------------------------------------------------------------
// NEAREST filter on the tensor cores.  The expansion
//   e(q, x) = |q|^2 + |x|^2 - 2 q.x
// is one contraction over D + 2 terms once the norms ride along as two extra
// coordinates: A[q] = (-2 q, 1, |q|^2) and B[x] = (x, |x|^2 (1 - kTc), 1),
// zero-padded to K.  A warp owns 32 queries (two 16-row m-tiles, A fragments
// in registers for the whole kernel) and walks the block's shared-memory
// vertex tile 8 vertices at a time with ldmatrix and mma.sync; the
// accumulators are the filter values, compared in registers against the
// running bound of their query.  Two operand types:
//
//  - FP16 for D + 2 <= 16 (nearest_tc16_kernel: one m16n8k16 per m-tile and
//    8 vertices).  The coordinates are first multiplied by a power of two 2^s
//    (exact), chosen from the largest coordinate magnitude of the batch so
//    that every scaled coordinate is below 16 and every scaled squared norm
//    below 256 D: the operands stay inside FP16's range.  Rounding to FP16
//    costs at most 2^-11 of an operand, or the operand itself when it is
//    below 2^-14 (a flush); with scaled coordinates below 16 the flushes add
//    less than 48 D 2^-14 + 2^-13 < kAbs = 2^-4 in all.
//  - TF32 for larger D (nearest_tc_kernel: m16n8k8 steps).  TF32 keeps 10 of
//    the 23 stored mantissa bits (truncation or rounding: 2^-10 of an
//    operand); there is no scaling, and every nonzero coordinate must lie in
//    [2^-60, 2^60] (normal products, no overflow).
//
// Products are exact and the FP32 accumulation error stays below 2^-14 of
// sum |a_k b_k| for K <= 32.  With sum |a_k b_k| <= 2 (|q|^2 + |x|^2) the
// computed value is within 1.0625 * 2^-9 (FP16; 1.04 * 2^-8 for TF32) of
// (|q|^2 + |x|^2), plus kAbs for FP16, from e (scaled units).  The vertex half
// of that error is taken out of B (kTc), the query half goes into the bound
// (kTq |q|^2).  The exact FP32 squared distance (sum of fmaf((q_d - x_d)^2))
// is within 4 (D + 2) u d^2 of the true one (u = 2^-24), so a bound built from
// the exact distance d2 of any admissible vertex as
//   lim = (d2 2^2s (1 + 4 (D + 2) u) + kTq |q|^2 + kAbs) (1 + 4 u)
// is never below the computed filter value of the true nearest vertex.  Every
// vertex that passes is re-evaluated with the exact formula on the unscaled
// FP32 coordinates, which alone decides: the results equal the plain scan's.
// The ordering pass flags inputs outside the operand type's range (NaN and
// infinities always) and the kernel then sends every pair to the exact check.
constexpr int kTcWarps = 8;
constexpr int kSliceAlign = 256;           // tree slices are whole tensor-core tiles
constexpr int kTcThreads = kTcWarps * 32;
constexpr int kTcQueries = kTcWarps * 32;  // queries per block
constexpr float kTc = 1.125f / 256.f;      // TF32: folded into |x|^2
constexpr float kTq = 1.25f / 256.f;       // TF32: widening by |q|^2
constexpr float kTc16 = 1.125f / 512.f;    // FP16: folded into |x|^2
constexpr float kTq16 = 1.25f / 512.f;     // FP16: widening by |q|^2
constexpr float kAbs16 = 1.f / 16.f;       // FP16: flushed operands (scaled units)

template <int DIM>
struct TcShape {
    static constexpr int K = ((DIM + 2 + 7) / 8) * 8;  // contraction length
    static constexpr int KS = K / 8;                   // m16n8k8 steps
    static constexpr int CH = K / 4;                   // 16-byte chunks per vertex row
    static constexpr int VT = K <= 16 ? 256 : 128;     // vertices per tile (16 KB)
};

// Chunk swizzle of a vertex row: the 8 rows one ldmatrix reads (8 consecutive
// vertices, one chunk each) land in 8 distinct 16-byte bank groups.
template <int CH>
__device__ __forceinline__ int tc_swz(int v) {
    if (CH == 8) return v & 7;
    if (CH == 4) return (v >> 1) & 3;
    return (v >> 2) & 1;  // CH = 2 or 6
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, "
        "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned &r0, unsigned &r1, unsigned &r2,
                                        unsigned &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr)
                 : "memory");
}
__device__ __forceinline__ void ldsm_x2(unsigned addr, unsigned &r0, unsigned &r1) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];"
                 : "=r"(r0), "=r"(r1)
                 : "r"(addr)
                 : "memory");
}

// Pieces shared by both filter kernels.
//
// Stage the block's kTcQueries queries (SoA rows of the ordered batch) in
// shared memory, one per thread (kTcThreads == kTcQueries).
template <int DIM>
__device__ __forceinline__ void tc_stage_queries(float (*qsm)[kTcQueries],
                                                 const float *__restrict__ queries, int Q, int qb) {
    const int j = threadIdx.x;
    const bool ok = qb + j < Q;
#pragma unroll
    for (int d = 0; d < DIM; ++d) qsm[d][j] = ok ? __ldg(queries + (size_t)d * Q + qb + j) : 0.f;
}

// Smallest g of the tree slice [vs, ve) (row DIM of the ordered tree), for
// every thread of the block: an admissible vertex of the slice has
// |q - x| < c - that minimum.
template <int DIM>
__device__ __forceinline__ float tc_slice_gmin(const float *__restrict__ tree, int ldt, int vs,
                                               int ve, float *red_g) {
    float gm = FLT_MAX;
#pragma unroll 4
    for (int v = vs + threadIdx.x; v < ve; v += kTcThreads)
        gm = fminf(gm, __ldg(tree + (size_t)DIM * ldt + v));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gm = fminf(gm, __shfl_xor_sync(kFull, gm, o));
    if ((threadIdx.x & 31) == 0) red_g[threadIdx.x >> 5] = gm;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kTcWarps; ++k) gm = fminf(gm, red_g[k]);
    return gm;
}

// The four lanes of a quad hold the same four rows (queries row_q(r)), each
// with the best of its own vertex columns, as a position in the g order:
// translate to original indices (perm), combine by key, and let lane
// tig == 0 write the slice's partial bests.
// Where a budget-ordered filter block finishes its query block: the slice
// blocks of query block b count themselves in qdone[b]; the last one to
// finish reduces the partial bests of every slice, best key first, and writes
// the original query's index.
struct NnFinish {
    int *qdone;            // [query blocks] slices finished (zero before the filter)
    const int *qperm;      // ordered query -> original query index
    int64_t *out_idx;      // [Q] by original query index
};

// No slice of the block has work (its cut is empty): no query of it has an
// admissible vertex.
__device__ __forceinline__ void nn_write_none(const NnFinish &fin, int qb, int Q) {
    for (int j = threadIdx.x; j < kTcQueries; j += blockDim.x)
        if (qb + j < Q) fin.out_idx[fin.qperm[qb + j]] = -1;
}

// Called by every thread of a slice block after its partial bests are
// written; ns = slice blocks of this query block that have work.
__device__ __forceinline__ void nn_finish(const Best *partial, const NnFinish &fin, int qblk,
                                          int ns, int qb, int Q) {
    __shared__ int s_last;
    __threadfence();  // this thread's partial records, before the count
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(fin.qdone + qblk, 1) == ns - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int j = threadIdx.x; j < kTcQueries; j += blockDim.x) {
        const int q = qb + j;
        if (q >= Q) continue;
        Best b{FLT_MAX * 2.f, FLT_MAX * 2.f, -1};
        for (int y = 0; y < ns; ++y) {
            const Best *rec = partial + (size_t)y * Q + q;
            const Best o{__ldcg(&rec->d2), __ldcg(&rec->g), __ldcg(&rec->idx)};
            if (better(o, b)) b = o;
        }
        fin.out_idx[fin.qperm[q]] = b.idx;
    }
}

template <typename RowQ>
__device__ __forceinline__ void tc_write_rows(Best (&best)[4], const int *__restrict__ perm,
                                              RowQ row_q, int Q, Best *__restrict__ partial) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if (best[r].idx >= 0) best[r].idx = __ldg(perm + best[r].idx);
#pragma unroll
        for (int o = 1; o <= 2; o <<= 1) {
            const Best other = shfl_best(best[r], o);
            if (better(other, best[r])) best[r] = other;
        }
        const int q = row_q(r);
        if ((threadIdx.x & 3) == 0 && q < Q) partial[(size_t)blockIdx.y * Q + q] = best[r];
    }
}

// Inputs: the g-ordered tree (SoA rows of stride ldt) with perm (ordered ->
// original index), the budget-ordered queries, cut (vertices each query block
// scans), the shared bound seed (see below); *exhaustive != 0 turns the filter
// off.  Block (x, y) takes query block b = gridDim.x - 1 - x (queries
// [256 b, 256 b + 256)) and the tree slice [y chunk, (y + 1) chunk) cut at
// cut[b]; its partial bests go to partial[y][q], and the query block's last
// slice block to finish reduces them (nn_finish).
template <int DIM>
__global__ void __launch_bounds__(kTcThreads)
nearest_tc_kernel(const float *__restrict__ tree, int N, int ldt, const float *__restrict__ queries,
                  const float *__restrict__ budgets, int Q, int chunk,
                  Best *__restrict__ partial, const int *__restrict__ perm,
                  const int *__restrict__ cut, float *__restrict__ seed,
                  const int *__restrict__ exhaustive, NnFinish fin) {
    using S = TcShape<DIM>;
    constexpr int K = S::K, KS = S::KS, CH = S::CH, VT = S::VT;
    __shared__ __align__(16) float xt[VT * K];  // vertex rows, swizzled chunks
    __shared__ float gt[VT];
    __shared__ float qsm[DIM][kTcQueries];      // the block's queries (exact checks)
    __shared__ float red_g[kTcWarps];
    constexpr float kU = 5.9604645e-8f;            // 2^-24
    constexpr float kC1 = 4.f * (DIM + 2.f) * kU;  // exact-distance relative error
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane >> 2, tig = lane & 3;
    // query blocks in descending budget order: the blocks with the longest
    // tree prefixes start first and the short ones fill the last wave
    const int qblk = gridDim.x - 1 - blockIdx.x;
    const int qb = qblk * kTcQueries;
    const int cut_q = min(N, cut[qblk]);
    const int vs = blockIdx.y * chunk;
    const int ve = min(cut_q, vs + chunk);
    if (vs >= ve) {  // no partial record: this slice is not counted
        if (blockIdx.y == 0) nn_write_none(fin, qb, Q);
        return;
    }
    const bool exact_only = *exhaustive != 0;

    tc_stage_queries<DIM>(qsm, queries, Q, qb);
    __syncthreads();
    // rows of this thread: slot r = 2 * mt + h is query qb + 32 warp + 16 mt + grp + 8 h
    auto row_l = [&](int r) { return warp * 32 + (r >> 1) * 16 + grp + (r & 1) * 8; };
    auto row_q = [&](int r) { return qb + row_l(r); };
    float cq[4], qn[4], lim[4];
    Best best[4];
    unsigned a[2][KS][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int q = row_q(r);
        const bool ok = q < Q;
        float n2 = 0.f;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const float v = qsm[d][row_l(r)];
            n2 = fmaf(v, v, n2);
        }
        qn[r] = n2;
        cq[r] = ok ? budgets[q] : -FLT_MAX;  // nothing is admissible for padding
        best[r] = Best{FLT_MAX * 2.f, FLT_MAX * 2.f, -1};
        lim[r] = FLT_MAX * 2.f;
    }
    // A fragments: a0 (row grp, k tig), a1 (row grp + 8, k tig), a2/a3 the same rows at k + 4
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = 2 * mt + (i & 1);
                const int q = row_q(r);
                const int k = 8 * ks + tig + 4 * (i >> 1);
                float v = 0.f;
                if (k < DIM)
                    v = q < Q ? -2.f * qsm[k][row_l(r)] : 0.f;
                else if (k == DIM)
                    v = 1.f;
                else if (k == DIM + 1)
                    v = qn[r];
                a[mt][ks][i] = __float_as_uint(v);
            }
        }
    }
    unsigned *const shared_lim = reinterpret_cast<unsigned *>(seed);
    auto widen = [&](int r, float sd) {
        if (sd <= FLT_MAX) lim[r] = fminf(lim[r], fmaf(sd, 1.f + kC1, kTq * qn[r]) * (1.f + 4.f * kU));
    };
    unsigned pend[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int q = row_q(r);
        pend[r] = q < Q ? __ldcg(shared_lim + q) : 0x7f800000u;
        widen(r, __uint_as_float(pend[r]));
    }
    {
        // an admissible vertex of this slice has |q - x| < c - g_min(slice)
        const float gm = tc_slice_gmin<DIM>(tree, ldt, vs, ve, red_g);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (!(cq[r] > gm)) {
                lim[r] = -FLT_MAX * 2.f;
            } else if (exact_only) {
                lim[r] = FLT_MAX * 2.f;
            } else {
                const float t = __fsub_ru(cq[r], gm);
                const float b2 = __fmul_ru(t, t);
                lim[r] = fminf(lim[r], fmaf(b2, 1.f + kC1, kTq * qn[r]) * (1.f + 4.f * kU));
            }
        }
    }
    const unsigned xt_s = (unsigned)__cvta_generic_to_shared(xt);
    // ldmatrix row addresses of this lane: matrix (lane >> 3) of a pair of
    // k-steps, vertex row (lane & 7) of the 8-vertex n-tile
    const int lrow = lane & 7, lmat = lane >> 3;
    // The next tile's vertex (coordinates and g) is loaded into registers
    // while the current tile is being scanned, so that the load latency
    // overlaps the tensor-core work; 32-bit element indices keep the per-row
    // offsets cheap (N (D + 1) < 2^31).
    const int t_ld = threadIdx.x & (VT - 1);  // VT < kTcThreads: two threads per row store the same values
    float px[DIM + 1];
    auto prefetch = [&](int v0n) {
        const bool ok = t_ld < min(VT, ve - v0n);
        const unsigned base = (unsigned)(v0n + t_ld);
#pragma unroll
        for (int d = 0; d <= DIM; ++d) px[d] = ok ? __ldg(tree + (base + (unsigned)d * (unsigned)ldt)) : 0.f;
        if (!ok) px[DIM] = FLT_MAX * 2.f;  // padding vertex: g = +inf
    };
    prefetch(vs);
    for (int v0 = vs; v0 < ve; v0 += VT) {
        const int nv = min(VT, ve - v0);
        __syncthreads();
        {
            // one vertex row per thread: coordinates, folded norm, 1, zero pad
            float *row = xt + t_ld * K;
            const int sw = tc_swz<CH>(t_ld);
            const bool ok = t_ld < nv;
            float x[K];
            float n2 = 0.f;
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                x[d] = px[d];
                n2 = fmaf(x[d], x[d], n2);
            }
            x[DIM] = ok ? n2 * (1.f - kTc) : FLT_MAX * 2.f;  // padding: never passes
            x[DIM + 1] = 1.f;
#pragma unroll
            for (int d = DIM + 2; d < K; ++d) x[d] = 0.f;
            gt[t_ld] = px[DIM];
            float4 *row4 = reinterpret_cast<float4 *>(row);
#pragma unroll
            for (int c = 0; c < CH; ++c)
                row4[c ^ sw] = make_float4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
        }
        __syncthreads();
        if (v0 + VT < ve) prefetch(v0 + VT);
        // refresh the bounds from the shared one (loaded a tile ago)
        if (!exact_only) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int q = row_q(r);
                widen(r, __uint_as_float(pend[r]));
                if (q < Q) pend[r] = __ldcg(shared_lim + q);
            }
        }
        const int ng = (nv + 7) >> 3;
        for (int nt = 0; nt < ng; ++nt) {
            const int vrow = nt * 8 + lrow;
            unsigned b[KS][2];
#pragma unroll
            for (int kp = 0; kp + 1 < KS; kp += 2) {
                const int c = 2 * kp + lmat;  // chunk of k-step kp (lmat 0, 1) or kp + 1 (2, 3)
                const unsigned addr = xt_s + (unsigned)((vrow * K + 4 * (c ^ tc_swz<CH>(vrow))) * 4);
                ldsm_x4(addr, b[kp][0], b[kp][1], b[kp + 1][0], b[kp + 1][1]);
            }
            if (KS & 1) {
                const int c = 2 * (KS - 1) + (lmat & 1);
                const unsigned addr = xt_s + (unsigned)((vrow * K + 4 * (c ^ tc_swz<CH>(vrow))) * 4);
                ldsm_x2(addr, b[KS - 1][0], b[KS - 1][1]);
            }
            float acc[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[mt][i] = 0.f;
#pragma unroll
                for (int ks = 0; ks < KS; ++ks) mma_tf32(acc[mt], a[mt][ks], b[ks][0], b[ks][1]);
            }
            // c0, c1: row grp, vertices 2 tig, 2 tig + 1; c2, c3: row grp + 8.
            // Without the bound (exact_only) every pair goes to the exact check.
            bool any = exact_only;
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int i = 0; i < 4; ++i) any |= acc[mt][i] <= lim[2 * mt + (i >> 1)];
            if (!__any_sync(kFull, any)) continue;
            unsigned pass = 0;
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    pass |= (exact_only || acc[mt][i] <= lim[2 * mt + (i >> 1)]) ? 1u << (4 * mt + i) : 0u;
            // survivors are rare: one copy of the exact check, with the row's
            // state selected and written back by value
            while (pass) {
                const int e = __ffs(pass) - 1;
                pass &= pass - 1;
                const int r = 2 * (e >> 2) + ((e >> 1) & 1);
                const int q = row_q(r);
                const int vl = nt * 8 + 2 * tig + (e & 1);
                if (q >= Q || vl >= nv) continue;
                float c_r = cq[0], q_r = qn[0], l_r = lim[0];
                Best b_r = best[0];
#pragma unroll
                for (int k = 1; k < 4; ++k)
                    if (r == k) { c_r = cq[k]; q_r = qn[k]; l_r = lim[k]; b_r = best[k]; }
                const float g = gt[vl];
                // a vertex with g >= c is never admissible
                if (!(g < c_r)) continue;
                const float *xr = xt + vl * K;
                const int sw = tc_swz<CH>(vl);
                float d2 = 0.f;
                const float *qp = &qsm[0][q - qb];
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    const float dq = qp[d * kTcQueries] - xr[4 * ((d >> 2) ^ sw) + (d & 3)];
                    d2 = fmaf(dq, dq, d2);
                }
                // filter of Alg. 2: g_v + |q - q_v| < c (strict); key (d^2, g, index).
                // The running best keeps the vertex's position in the g order;
                // original indices (perm) are looked up only to break an exact
                // (d^2, g) tie, and once per row at the end.
                const int pos = v0 + vl;
                if (d2 <= b_r.d2 && g + __fsqrt_rn(d2) < c_r &&
                    (d2 < b_r.d2 || g < b_r.g ||
                     (g == b_r.g && __ldg(perm + pos) < __ldg(perm + b_r.idx)))) {
                    b_r = Best{d2, g, pos};
                    if (!exact_only) {
                        l_r = fminf(l_r, fmaf(d2, 1.f + kC1, kTq * q_r) * (1.f + 4.f * kU));
                        atomicMin(shared_lim + q, __float_as_uint(d2));
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (r == k) { lim[k] = l_r; best[k] = b_r; }
                }
            }
            // the quad's lanes scan different vertex columns of the same
            // rows: a record of one tightens the bound of all four
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                lim[r] = fminf(lim[r], __shfl_xor_sync(kFull, lim[r], 1));
                lim[r] = fminf(lim[r], __shfl_xor_sync(kFull, lim[r], 2));
            }
        }
    }
    tc_write_rows(best, perm, row_q, Q, partial);
    nn_finish(partial, fin, qblk, (cut_q + chunk - 1) / chunk, qb, Q);
}

__device__ __forceinline__ void mma_f16(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                        unsigned b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, "
        "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned pack_half2(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);  // lo in the low 16 bits
    return *reinterpret_cast<const unsigned *>(&h);
}

// FP16 form of the filter for D + 2 <= 16 (K = 16: one m16n8k16 per m-tile
// and 8 vertices; two groups of 8 vertices per ldmatrix.x4).  Same inputs as
// nearest_tc_kernel plus the ordering pass's largest coordinate magnitude
// (*maxabs, as float bits) and its non-finite flag (*nonfinite).  Vertex rows
// hold 16 halves (32 bytes, two 16-byte chunks swizzled by bit 2 of the
// vertex); the unscaled FP32 coordinates of the tile are kept beside them
// (SoA) for the exact checks.
// Registers are capped so that 3 blocks (24 warps) stay resident per SM.
template <int DIM>
__global__ void __launch_bounds__(kTcThreads, 3)
nearest_tc16_kernel(const float *__restrict__ tree, int N, int ldt, const float *__restrict__ queries,
                    const float *__restrict__ budgets, int Q, int chunk,
                    Best *__restrict__ partial, const int *__restrict__ perm,
                    const int *__restrict__ cut, float *__restrict__ seed,
                    const unsigned *__restrict__ maxabs, const int *__restrict__ nonfinite,
                    NnFinish fin) {
    static_assert(DIM + 2 <= 16, "FP16 filter holds K = 16");
    constexpr int VT = kTcThreads;                   // vertices per tile
    __shared__ __align__(16) unsigned xh[VT * 8];    // FP16 rows, swizzled chunks
    __shared__ float xf[DIM][VT];                    // unscaled FP32 coordinates
    __shared__ float gt[VT];
    __shared__ float qsm[DIM][kTcQueries];           // the block's queries (exact checks)
    __shared__ float red_g[kTcWarps];
    constexpr float kU = 5.9604645e-8f;            // 2^-24
    constexpr float kC1 = 4.f * (DIM + 2.f) * kU;  // exact-distance relative error
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane >> 2, tig = lane & 3;
    // query blocks in descending budget order: the blocks with the longest
    // tree prefixes start first and the short ones fill the last wave
    const int qblk = gridDim.x - 1 - blockIdx.x;
    const int qb = qblk * kTcQueries;
    const int cut_q = min(N, cut[qblk]);
    const int vs = blockIdx.y * chunk;
    const int ve = min(cut_q, vs + chunk);
    if (vs >= ve) {  // no partial record: this slice is not counted
        if (blockIdx.y == 0) nn_write_none(fin, qb, Q);
        return;
    }

    // power-of-two scale: largest magnitude in [2^(ex-1), 2^ex) -> [8, 16)
    int ex = 0;
    frexpf(__uint_as_float(*maxabs), &ex);
    const int sh = 4 - ex;
    const bool exact_only = *nonfinite != 0 || sh > 126;
    const float sc = exact_only ? 1.f : ldexpf(1.f, sh);

    tc_stage_queries<DIM>(qsm, queries, Q, qb);
    __syncthreads();
    auto row_l = [&](int r) { return warp * 32 + (r >> 1) * 16 + grp + (r & 1) * 8; };
    auto row_q = [&](int r) { return qb + row_l(r); };
    float cq[4], qs2[4], lim[4];  // qs2: scaled |q|^2
    Best best[4];
    unsigned a[2][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int q = row_q(r);
        float n2 = 0.f;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const float v = qsm[d][row_l(r)] * sc;
            n2 = fmaf(v, v, n2);
        }
        qs2[r] = n2;
        cq[r] = q < Q ? budgets[q] : -FLT_MAX;  // nothing is admissible for padding
        best[r] = Best{FLT_MAX * 2.f, FLT_MAX * 2.f, -1};
        lim[r] = FLT_MAX * 2.f;
    }
    // A fragments (16 x 16, row-major): register i holds row grp + 8 (i & 1),
    // columns 2 tig + 8 (i >> 1) and the next one
    auto a_val = [&](int r, int k) {
        if (k < DIM) return -2.f * (qsm[k][row_l(r)] * sc);
        if (k == DIM) return 1.f;
        if (k == DIM + 1) return qs2[r];
        return 0.f;
    };
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = 2 * mt + (i & 1), k = 2 * tig + 8 * (i >> 1);
            a[mt][i] = pack_half2(a_val(r, k), a_val(r, k + 1));
        }
    unsigned *const shared_lim = reinterpret_cast<unsigned *>(seed);
    // bound from the exact (unscaled) squared distance of an admissible vertex
    auto bound = [&](int r, float d2) {
        return fmaf((d2 * sc) * sc, 1.f + kC1, fmaf(kTq16, qs2[r], kAbs16)) * (1.f + 4.f * kU);
    };
    auto widen = [&](int r, float sd) {
        if (sd <= FLT_MAX) lim[r] = fminf(lim[r], bound(r, sd));
    };
    unsigned pend[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int q = row_q(r);
        pend[r] = q < Q ? __ldcg(shared_lim + q) : 0x7f800000u;
        widen(r, __uint_as_float(pend[r]));
    }
    {
        // an admissible vertex of this slice has |q - x| < c - g_min(slice)
        const float gm = tc_slice_gmin<DIM>(tree, ldt, vs, ve, red_g);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (!(cq[r] > gm)) {
                lim[r] = -FLT_MAX * 2.f;
            } else if (exact_only) {
                lim[r] = FLT_MAX * 2.f;
            } else {
                const float t = __fsub_ru(cq[r], gm);
                lim[r] = fminf(lim[r], bound(r, __fmul_ru(t, t)));
            }
        }
    }
    const unsigned xh_s = (unsigned)__cvta_generic_to_shared(xh);
    // ldmatrix.x4 row address of this lane: matrix lane >> 3 = (group of 8
    // vertices lane >> 4, chunk (lane >> 3) & 1), vertex row lane & 7
    const int lrow = lane & 7, lchunk = (lane >> 3) & 1, lgrp = lane >> 4;
    // next tile's vertex of this thread, loaded while the current one is scanned
    const int t_ld = threadIdx.x;
    float px[DIM + 1];
    auto prefetch = [&](int v0n) {
        const bool ok = t_ld < min(VT, ve - v0n);
        const unsigned base = (unsigned)(v0n + t_ld);
#pragma unroll
        for (int d = 0; d <= DIM; ++d) px[d] = ok ? __ldg(tree + (base + (unsigned)d * (unsigned)ldt)) : 0.f;
        if (!ok) px[DIM] = FLT_MAX * 2.f;  // padding vertex: g = +inf
    };
    prefetch(vs);
    for (int v0 = vs; v0 < ve; v0 += VT) {
        const int nv = min(VT, ve - v0);
        __syncthreads();
        {
            const bool ok = t_ld < nv;
            float h[16];
            float n2 = 0.f;
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                xf[d][t_ld] = px[d];
                h[d] = px[d] * sc;
                n2 = fmaf(h[d], h[d], n2);
            }
            h[DIM] = ok ? n2 * (1.f - kTc16) : FLT_MAX * 2.f;  // padding: never passes
            h[DIM + 1] = 1.f;
#pragma unroll
            for (int d = DIM + 2; d < 16; ++d) h[d] = 0.f;
            gt[t_ld] = px[DIM];
            uint4 *row = reinterpret_cast<uint4 *>(xh + t_ld * 8);
            const int sw = (t_ld >> 2) & 1;
            row[0 ^ sw] = make_uint4(pack_half2(h[0], h[1]), pack_half2(h[2], h[3]),
                                     pack_half2(h[4], h[5]), pack_half2(h[6], h[7]));
            row[1 ^ sw] = make_uint4(pack_half2(h[8], h[9]), pack_half2(h[10], h[11]),
                                     pack_half2(h[12], h[13]), pack_half2(h[14], h[15]));
        }
        __syncthreads();
        if (v0 + VT < ve) prefetch(v0 + VT);
        if (!exact_only) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int q = row_q(r);
                widen(r, __uint_as_float(pend[r]));
                if (q < Q) pend[r] = __ldcg(shared_lim + q);
            }
        }
        const int ng2 = (nv + 15) >> 4;  // pairs of 8-vertex groups
#pragma unroll 2
        for (int np = 0; np < ng2; ++np) {
            const int vrow = (2 * np + lgrp) * 8 + lrow;
            unsigned b[2][2];
            ldsm_x4(xh_s + (unsigned)(vrow * 32 + 16 * (lchunk ^ ((vrow >> 2) & 1))), b[0][0],
                    b[0][1], b[1][0], b[1][1]);
            float acc[2][2][4];
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) acc[j][mt][i] = 0.f;
                    mma_f16(acc[j][mt], a[mt], b[j][0], b[j][1]);
                }
            // element (j, mt, i): row grp + 8 (i >> 1) of m-tile mt, vertex
            // 8 (2 np + j) + 2 tig + (i & 1)
            // the common case, nothing passes: one compare per row on the
            // minimum of its four values (a NaN never passes either way)
            bool any = exact_only;
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float m = fminf(fminf(acc[0][mt][2 * h], acc[0][mt][2 * h + 1]),
                                          fminf(acc[1][mt][2 * h], acc[1][mt][2 * h + 1]));
                    any |= m <= lim[2 * mt + h];
                }
            if (!__any_sync(kFull, any)) continue;
            unsigned pass = 0;
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        pass |= (exact_only || acc[j][mt][i] <= lim[2 * mt + (i >> 1)])
                                    ? 1u << (8 * j + 4 * mt + i) : 0u;
            while (pass) {
                const int e = __ffs(pass) - 1;
                pass &= pass - 1;
                const int r = 2 * ((e >> 2) & 1) + ((e >> 1) & 1);
                const int q = row_q(r);
                const int vl = (2 * np + (e >> 3)) * 8 + 2 * tig + (e & 1);
                if (q >= Q || vl >= nv) continue;
                float c_r = cq[0], l_r = lim[0];
                Best b_r = best[0];
#pragma unroll
                for (int k = 1; k < 4; ++k)
                    if (r == k) { c_r = cq[k]; l_r = lim[k]; b_r = best[k]; }
                const float g = gt[vl];
                // a vertex with g >= c is never admissible
                if (!(g < c_r)) continue;
                float d2 = 0.f;
                const float *qp = &qsm[0][q - qb];
                const float *xp = &xf[0][vl];
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    const float dq = qp[d * kTcQueries] - xp[d * VT];
                    d2 = fmaf(dq, dq, d2);
                }
                // filter of Alg. 2: g_v + |q - q_v| < c (strict); key (d^2, g, index).
                // The running best keeps the vertex's position in the g order;
                // original indices (perm) are looked up only to break an exact
                // (d^2, g) tie, and once per row at the end.
                const int pos = v0 + vl;
                if (d2 <= b_r.d2 && g + __fsqrt_rn(d2) < c_r &&
                    (d2 < b_r.d2 || g < b_r.g ||
                     (g == b_r.g && __ldg(perm + pos) < __ldg(perm + b_r.idx)))) {
                    b_r = Best{d2, g, pos};
                    if (!exact_only) {
                        float bq = 0.f;
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            if (r == k) bq = bound(k, d2);
                        l_r = fminf(l_r, bq);
                        atomicMin(shared_lim + q, __float_as_uint(d2));
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (r == k) { lim[k] = l_r; best[k] = b_r; }
                }
            }
            // the quad's lanes scan different vertex columns of the same
            // rows: a record of one tightens the bound of all four
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                lim[r] = fminf(lim[r], __shfl_xor_sync(kFull, lim[r], 1));
                lim[r] = fminf(lim[r], __shfl_xor_sync(kFull, lim[r], 2));
            }
        }
    }
    tc_write_rows(best, perm, row_q, Q, partial);
    nn_finish(partial, fin, qblk, (cut_q + chunk - 1) / chunk, qb, Q);
}

// ---------------------------------------------------------------------------
// NEAREST filter in FP32 on the FMA pipe (the default for large batches).
// The same expansion as the tensor-core filters, e(q, x) = |q|^2 + |x|^2 -
// 2 q.x, is computed per (query, vertex) pair as a chain of D fused
// multiply-adds that starts from the vertex's folded squared norm:
//   acc = xn + sum_d (-2 q_d) x_d,   xn = fl(|x|^2) (1 - 4 gamma),
// and a pair passes when acc <= T_q, a per-query threshold with |q|^2 taken
// out.  The ordering pass stores xn as an extra row of the ordered tree.  A
// thread owns 8 queries x 8 vertices of each 64-vertex step (a register tile
// of 64 accumulators); the operands are read as 16-byte vectors from
// dimension-major shared arrays, every load a broadcast or one conflict-free
// row.  For 8 <= D <= 21 the tile is updated with packed FP32 FMAs (fma.rn.f32x2:
// two IEEE single-precision FMAs per instruction, each rounded as fmaf, so
// the accumulators are bit-identical to the scalar chain): the multipliers
// -2 q_d are kept twice in shared memory, {a, a}, and pair with two adjacent
// vertex columns, 6 shared loads per 32 packed FMAs (64 FMAs).  That halves
// the instructions the FMA chain issues; the pipe's FMA rate is unchanged, so
// the other instructions of the scan fit in the issue slots it frees.  Warp
// lanes 8 ty' + tx share the queries of ty (8 lanes) and the vertex columns
// of tx.  Tree tiles come in by cp.async
// into a double buffer, one barrier per tile; the running best of each
// (thread, query) sits in shared memory and is touched only when a pair
// passes, so that two blocks (16 warps) stay resident per SM.
//
// Error bound (u = 2^-24, gamma = kF32G (D + 2) = 1.25 (D + 2) u; the ordering
// pass sends every pair to the exact check unless every nonzero coordinate
// lies in [2^-60, 2^60], so no product or squared norm over- or underflows):
//   * fl(|x|^2) is within gamma |x|^2, so xn + gamma (xn + |x|^2) <= |x|^2;
//   * the chain adds at most gamma (xn + sum |2 q_d x_d|) <=
//     gamma (xn + |q|^2 + |x|^2), hence acc <= |q - x|^2 - |q|^2 (1 - gamma);
//   * qn = fl(|q|^2) is within gamma |q|^2, hence acc <= |q - x|^2 - qn +
//     2 gamma qn.
// The exact formula's d2 of any admissible vertex is at least |q - x*|^2 /
// (1 + kC1) for the true nearest admissible x* (kC1 = 4 (D + 2) u), so
//   T_q = fl_up( fl(fmaf(d2, 1 + kC1, 2 gamma qn)) (1 + 4 u) - qn )
// satisfies acc(x*) <= T_q: the filter never drops the true nearest vertex.
// Every vertex that passes is decided by the exact formula on the FP32
// coordinates, so the results equal the plain scan's, ties included.
// ---------------------------------------------------------------------------
constexpr float kF32G = 1.25f * 5.9604645e-8f;  // gamma / (D + 2)
constexpr int kF32Step = 64;                     // vertices per register-tile step

template <int DIM>
struct F32Shape {
    // packed FMAs (the multipliers kept twice) where two blocks still fit and
    // the tile's registers do not spill (they do below 8 dimensions)
    static constexpr bool PACKED = DIM >= 8 && DIM <= 21;
    // vertices per shared-memory tile (six 64-vertex steps per barrier up to
    // 14 dimensions) such that two blocks of 256 threads fit an SM
    static constexpr int VT = DIM <= 14 ? 384 : (DIM <= 21 && !PACKED) ? 128 : 64;
    static constexpr int ROWS = DIM + 2;              // x_d, g, folded |x|^2
    static constexpr int AM = PACKED ? 2 : 1;         // copies of each -2 q_d
};

template <int DIM>
constexpr size_t f32_smem_bytes() {
    // -2 q [DIM][256] (twice when packed), two tiles [ROWS][VT], best d2,
    // best position and bound [8][256] each
    return sizeof(float) * ((size_t)F32Shape<DIM>::AM * DIM * kTcQueries +
                            (size_t)2 * F32Shape<DIM>::ROWS * F32Shape<DIM>::VT +
                            (size_t)3 * 8 * kTcQueries);
}

// Smallest of three floats (a NaN input is ignored while another is not NaN).
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

typedef unsigned long long f32x2_t;  // two floats, the first in the low half

__device__ __forceinline__ f32x2_t fma_f32x2(f32x2_t a, f32x2_t b, f32x2_t c) {
    f32x2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ float f32x2_lo(f32x2_t v) { return __uint_as_float((unsigned)v); }
__device__ __forceinline__ float f32x2_hi(f32x2_t v) {
    return __uint_as_float((unsigned)(v >> 32));
}

// Source of the padding columns' folded norms: +inf never passes the filter.
__device__ const float g_f32_pad_inf = __builtin_inff();

__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool ok) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src),
                 "r"(ok ? 4 : 0)
                 : "memory");
}
// 16 bytes, of which the first src_bytes come from global memory and the
// rest are zero (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(float *dst, const float *src, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int DIM>
__global__ void __launch_bounds__(kTcThreads, 2)
nearest_f32_kernel(const float *__restrict__ tree, int N, int ldt, const float *__restrict__ queries,
                   const float *__restrict__ budgets, int Q, int chunk,
                   Best *__restrict__ partial, const int *__restrict__ perm,
                   const int *__restrict__ cut, float *__restrict__ seed,
                   const int *__restrict__ exact_only_flag, NnFinish fin) {
    constexpr int VT = F32Shape<DIM>::VT, ROWS = F32Shape<DIM>::ROWS, AM = F32Shape<DIM>::AM;
    extern __shared__ __align__(16) float f32_sm[];
    // -2 q_d of query j at am[d][AM j .. AM j + AM - 1]
    float(*am)[AM * kTcQueries] = reinterpret_cast<float(*)[AM * kTcQueries]>(f32_sm);
    float *tiles = f32_sm + AM * DIM * kTcQueries;                // [2][ROWS][VT]
    float(*sb_d2)[kTcQueries] =
        reinterpret_cast<float(*)[kTcQueries]>(tiles + 2 * ROWS * VT);  // [8][256]
    int(*sb_pos)[kTcQueries] = reinterpret_cast<int(*)[kTcQueries]>(sb_d2 + 8);
    float(*lim_s)[kTcQueries] = reinterpret_cast<float(*)[kTcQueries]>(sb_pos + 8);
    __shared__ float qn_s[kTcQueries];                   // fl(|q|^2)
    __shared__ float cq_s[kTcQueries];                   // budgets
    __shared__ unsigned sl_s[kTcQueries];                // shared bounds, one tile old
    __shared__ float red_g[kTcWarps];
    constexpr float kU = 5.9604645e-8f;                   // 2^-24
    constexpr float kC1 = 4.f * (DIM + 2.f) * kU;         // exact-distance relative error
    constexpr float kG = kF32G * (DIM + 2.f);             // gamma
    const int tid = threadIdx.x;
    const int ty = tid >> 3, tx = tid & 7;
    // query blocks in descending budget order: the blocks with the longest
    // tree prefixes start first and the short ones fill the last wave
    const int qblk = gridDim.x - 1 - blockIdx.x;
    const int qb = qblk * kTcQueries;
    const int cut_q = min(N, cut[qblk]);
    const int vs = blockIdx.y * chunk;
    const int ve = min(cut_q, vs + chunk);
    if (vs >= ve) {  // no partial record: this slice is not counted
        if (blockIdx.y == 0) nn_write_none(fin, qb, Q);
        return;
    }
    const bool exact_only = *exact_only_flag != 0;
    unsigned *const shared_lim = reinterpret_cast<unsigned *>(seed);

    // first tile in flight while the queries are staged
    // 16-byte pieces (rows start on 16-byte boundaries, slices and tiles on
    // multiples of 4 vertices); a piece past the slice end is zero-filled, its
    // folded norms +inf so that the padding columns never pass
    auto issue_tile = [&](int v0n, int buf) {
        const int nvn = min(VT, ve - v0n);
        float *dst = tiles + buf * ROWS * VT;
        for (int i = tid; i < ROWS * (VT / 4); i += kTcThreads) {
            const int d = i / (VT / 4), j = 4 * (i - d * (VT / 4));
            float *to = dst + d * VT + j;
            const float *from = tree + ((size_t)d * ldt + v0n + j);
            if (j + 4 <= nvn) {
                cp_async16(to, from, 16);
            } else if (d == DIM + 1) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    cp_async4(to + k, j + k < nvn ? from + k : &g_f32_pad_inf, true);
            } else {
                cp_async16(to, j < nvn ? from : tree, 4 * max(0, nvn - j));
            }
        }
        cp_async_commit();
    };
    issue_tile(vs, 0);

    // The queries themselves are not kept: within the filter's coordinate
    // range [2^-60, 2^60] both -2 q_d and -0.5 (-2 q_d) are exact, so the exact
    // check takes q_d back from the multipliers; in exact-only mode it reads
    // the ordered queries from global memory instead.
    {
        const int j = tid;
        const bool ok = qb + j < Q;
        float n2 = 0.f;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const float v = ok ? __ldg(queries + (size_t)d * Q + qb + j) : 0.f;
            const float a = -2.f * v;
            if constexpr (AM == 2)
                *reinterpret_cast<float2 *>(&am[d][2 * j]) = make_float2(a, a);
            else
                am[d][j] = a;
            n2 = fmaf(v, v, n2);
        }
        qn_s[j] = n2;
        cq_s[j] = qb + j < Q ? budgets[qb + j] : -FLT_MAX;  // padding admits nothing
        sl_s[j] = qb + j < Q ? __ldcg(shared_lim + qb + j) : 0x7f800000u;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            sb_d2[r][j] = FLT_MAX * 2.f;
            sb_pos[r][j] = -1;
        }
    }
    __syncthreads();
    // row r of this thread: query ql(r) of the block; rows of real queries
    auto ql = [&](int r) { return r < 4 ? ty * 4 + r : 128 + ty * 4 + (r - 4); };
    unsigned row_ok = 0;
#pragma unroll
    for (int r = 0; r < 8; ++r) row_ok |= qb + ql(r) < Q ? 1u << r : 0u;
    auto bound = [&](int r, float d2) {
        const float qn = qn_s[ql(r)];
        return __fsub_ru(fmaf(d2, 1.f + kC1, 2.f * kG * qn) * (1.f + 4.f * kU), qn);
    };
    float lim[8];
    {
        // an admissible vertex of this slice has |q - x| < c - g_min(slice)
        const float gm = tc_slice_gmin<DIM>(tree, ldt, vs, ve, red_g);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const float c = cq_s[ql(r)];
            if (!(c > gm)) {
                lim[r] = -FLT_MAX * 2.f;
            } else if (exact_only) {
                lim[r] = FLT_MAX * 2.f;
            } else {
                const float t = __fsub_ru(c, gm);
                lim[r] = bound(r, __fmul_ru(t, t));
            }
        }
    }
    unsigned sl_next = 0x7f800000u;  // this thread's query tid, for the next tile
    int buf = 0;
    for (int v0 = vs; v0 < ve; v0 += VT, buf ^= 1) {
        const int nv = min(VT, ve - v0);
        const float(*xs)[VT] = reinterpret_cast<const float(*)[VT]>(tiles + buf * ROWS * VT);
        cp_async_wait_all();
        // (a newer bound than another thread's view is still a valid bound)
        if (v0 > vs) sl_s[tid] = sl_next;
        __syncthreads();  // tile visible; every thread is done with the other buffer
        if (v0 + VT < ve) issue_tile(v0 + VT, buf ^ 1);
        if (qb + tid < Q) sl_next = __ldcg(shared_lim + qb + tid);
        if (!exact_only) {
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const float sd = __uint_as_float(sl_s[ql(r)]);
                if (sd <= FLT_MAX) lim[r] = fminf(lim[r], bound(r, sd));
            }
        }
        const int steps = (nv + kF32Step - 1) / kF32Step;
        for (int s = 0; s < steps; ++s) {
            const int c0 = s * kF32Step + tx * 4;  // columns c0..c0+3 and c0+32..c0+35
            float acc[8][8];
            if constexpr (AM == 2) {
                // pairs of adjacent columns: p = 0, 1 -> c0 + 2p, 2 -> c0 + 32, 3 -> c0 + 34
                const ulonglong2 n0 = *reinterpret_cast<const ulonglong2 *>(&xs[DIM + 1][c0]);
                const ulonglong2 n1 = *reinterpret_cast<const ulonglong2 *>(&xs[DIM + 1][c0 + 32]);
                const f32x2_t xn[4] = {n0.x, n0.y, n1.x, n1.y};
                f32x2_t acc2[8][4];
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    // {a, a} of rows 0-1, 2-3 (queries 4 ty ..) and 4-5, 6-7 (128 + 4 ty ..)
                    const ulonglong2 a0 = *reinterpret_cast<const ulonglong2 *>(&am[d][8 * ty]);
                    const ulonglong2 a1 = *reinterpret_cast<const ulonglong2 *>(&am[d][8 * ty + 4]);
                    const ulonglong2 a2 =
                        *reinterpret_cast<const ulonglong2 *>(&am[d][256 + 8 * ty]);
                    const ulonglong2 a3 =
                        *reinterpret_cast<const ulonglong2 *>(&am[d][256 + 8 * ty + 4]);
                    const ulonglong2 x0 = *reinterpret_cast<const ulonglong2 *>(&xs[d][c0]);
                    const ulonglong2 x1 = *reinterpret_cast<const ulonglong2 *>(&xs[d][c0 + 32]);
                    const f32x2_t a[8] = {a0.x, a0.y, a1.x, a1.y, a2.x, a2.y, a3.x, a3.y};
                    const f32x2_t x[4] = {x0.x, x0.y, x1.x, x1.y};
#pragma unroll
                    for (int r = 0; r < 8; ++r)
#pragma unroll
                        for (int p = 0; p < 4; ++p)
                            acc2[r][p] = fma_f32x2(a[r], x[p], d == 0 ? xn[p] : acc2[r][p]);
                }
#pragma unroll
                for (int r = 0; r < 8; ++r)
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        acc[r][2 * p] = f32x2_lo(acc2[r][p]);
                        acc[r][2 * p + 1] = f32x2_hi(acc2[r][p]);
                    }
            } else {
                const float4 n0 = *reinterpret_cast<const float4 *>(&xs[DIM + 1][c0]);
                const float4 n1 = *reinterpret_cast<const float4 *>(&xs[DIM + 1][c0 + 32]);
                const float xn[8] = {n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, n1.z, n1.w};
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    const float4 a0 = *reinterpret_cast<const float4 *>(&am[d][ty * 4]);
                    const float4 a1 = *reinterpret_cast<const float4 *>(&am[d][128 + ty * 4]);
                    const float4 x0 = *reinterpret_cast<const float4 *>(&xs[d][c0]);
                    const float4 x1 = *reinterpret_cast<const float4 *>(&xs[d][c0 + 32]);
                    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                    const float x[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                    for (int r = 0; r < 8; ++r)
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            acc[r][c] = fmaf(a[r], x[c], d == 0 ? xn[c] : acc[r][c]);
                }
            }
            // the common case, nothing passes: one compare per row on the
            // minimum of its eight values (a NaN never passes either way);
            // rows of padding queries (q >= Q) never pass
            unsigned rows = 0;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const float m = fmin3(fmin3(acc[r][0], acc[r][1], acc[r][2]),
                                      fmin3(acc[r][3], acc[r][4], acc[r][5]),
                                      fminf(acc[r][6], acc[r][7]));
                rows |= (exact_only || m <= lim[r]) ? 1u << r : 0u;
            }
            rows &= row_ok;
            if (!__any_sync(kFull, rows != 0u)) continue;
            // pass bits r * 8 + c of the rows that pass, then one loop over
            // them with the bounds in shared memory (dynamic row index)
            unsigned long long pass = 0ull;
#pragma unroll
            for (int r = 0; r < 8; ++r)
                if ((rows >> r) & 1u) {
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        if (exact_only || acc[r][c] <= lim[r]) pass |= 1ull << (8 * r + c);
                }
            if (pass) {
#pragma unroll
                for (int r = 0; r < 8; ++r) lim_s[r][tid] = lim[r];
#pragma unroll 1
                while (pass) {
                    const int bit = __ffsll((long long)pass) - 1;
                    pass &= pass - 1;
                    const int r = bit >> 3, c = bit & 7;
                    const int vl = c0 + (c < 4 ? c : 28 + c);
                    if (vl >= nv) continue;
                    const float g = xs[DIM][vl];
                    const int qlr = r < 4 ? ty * 4 + r : 128 + ty * 4 + (r - 4);
                    const float cr = cq_s[qlr];
                    // a vertex with g >= c is never admissible
                    if (!(g < cr)) continue;
                    float d2 = 0.f;
                    if (exact_only) {
#pragma unroll
                        for (int d = 0; d < DIM; ++d) {
                            const float dq = __ldg(queries + (size_t)d * Q + qb + qlr) - xs[d][vl];
                            d2 = fmaf(dq, dq, d2);
                        }
                    } else {
#pragma unroll
                        for (int d = 0; d < DIM; ++d) {
                            // one rounding of q_d - x_d, as the plain difference
                            const float dq = fmaf(-0.5f, am[d][AM * qlr], -xs[d][vl]);
                            d2 = fmaf(dq, dq, d2);
                        }
                    }
                    // filter of Alg. 2: g_v + |q - q_v| < c (strict); key (d^2,
                    // g, index), the running best keeps the vertex's position in
                    // the g order (its g is looked up there; original indices
                    // break exact ties)
                    const float bd2 = sb_d2[r][tid];
                    if (!(d2 <= bd2) || !(g + __fsqrt_rn(d2) < cr)) continue;
                    const int bpos = sb_pos[r][tid];
                    bool take = d2 < bd2 || bpos < 0;
                    if (!take) {
                        const float bg = __ldg(tree + (size_t)DIM * ldt + bpos);
                        take = g < bg || (g == bg && __ldg(perm + v0 + vl) < __ldg(perm + bpos));
                    }
                    if (take) {
                        sb_d2[r][tid] = d2;
                        sb_pos[r][tid] = v0 + vl;
                        if (!exact_only) {
                            const float qn = qn_s[qlr];
                            const float bq = __fsub_ru(
                                fmaf(d2, 1.f + kC1, 2.f * kG * qn) * (1.f + 4.f * kU), qn);
                            lim_s[r][tid] = fminf(lim_s[r][tid], bq);
                            atomicMin(shared_lim + qb + qlr, __float_as_uint(d2));
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < 8; ++r) lim[r] = lim_s[r][tid];
            }
            // the 8 lanes of a query group scan different vertex columns of
            // the same rows: a record of one tightens the bound of all
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                lim[r] = fminf(lim[r], __shfl_xor_sync(kFull, lim[r], 1));
                lim[r] = fminf(lim[r], __shfl_xor_sync(kFull, lim[r], 2));
                lim[r] = fminf(lim[r], __shfl_xor_sync(kFull, lim[r], 4));
            }
        }
    }
    // original indices, then the best of the query group's 8 lanes
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int pos = sb_pos[r][tid];
        Best b{FLT_MAX * 2.f, FLT_MAX * 2.f, -1};
        if (pos >= 0) b = Best{sb_d2[r][tid], __ldg(tree + (size_t)DIM * ldt + pos), __ldg(perm + pos)};
#pragma unroll
        for (int o = 1; o <= 4; o <<= 1) {
            const Best other = shfl_best(b, o);
            if (better(other, b)) b = other;
        }
        const int q = qb + ql(r);
        if (tx == 0 && q < Q) partial[(size_t)blockIdx.y * Q + q] = b;
    }
    nn_finish(partial, fin, qblk, (cut_q + chunk - 1) / chunk, qb, Q);
}

// ---------------------------------------------------------------------------
// Budget-ordered NEAREST for large batches.  A vertex with g_v >= c is never
// admissible (distances are >= 0), so once the tree is ordered by g and the
// queries by budget, a block of queries only needs the prefix of the tree
// whose g lies below its largest budget.  Both orders come from counting
// sorts into kSortBuckets buckets over the finite range of g (budgets are
// bucketed on the same scale); the order inside a bucket does not matter,
// because exact ties are broken by original vertex index.
// ---------------------------------------------------------------------------
constexpr int kSortBuckets = 1024;

struct SortState {
    int gmin, gmax;                      // order-preserving keys of the finite g range
    int exact_only;                      // a coordinate lies outside the TF32 filter's range
    int nonfinite;                       // a coordinate is NaN or infinite
    unsigned maxabs;                     // largest finite coordinate magnitude (float bits)
    int arrive;                          // histogram blocks done (the last one scans)
    int tree_off[kSortBuckets + 1];      // bucket starts of the g-ordered tree
    int tree_cur[kSortBuckets];
    int query_off[kSortBuckets + 1];
    int query_cur[kSortBuckets];
};

__device__ __forceinline__ int fkey(float v) {
    const int k = __float_as_int(v);
    return k ^ ((k >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float unkey(int o) { return __int_as_float(o ^ ((o >> 31) & 0x7fffffff)); }

// Bucket of a value on the g scale; monotonic in v (a subtraction and a
// product by a positive constant), non-finite values go to the last bucket.
__device__ __forceinline__ int sort_bucket(float v, float lo, float scale) {
    if (!(fabsf(v) <= FLT_MAX)) return kSortBuckets - 1;
    const float b = floorf((v - lo) * scale);
    if (!(b > 0.f)) return 0;
    return b >= (float)(kSortBuckets - 1) ? kSortBuckets - 1 : (int)b;
}

__device__ __forceinline__ void g_scale(const SortState &S, float *lo, float *scale) {
    const float a = unkey(S.gmin), b = unkey(S.gmax);
    *lo = a;
    *scale = b > a ? (float)kSortBuckets / (b - a) : 0.f;
}

// First pass of a call: resets the sort state and the filter's per-query-block
// slice counters, and (with_range) finds the finite range of g in the same
// single block; larger trees take sort_range after it.
constexpr int kSetupThreads = 1024;
constexpr int kSetupRangeMax = 1 << 17;  // largest N whose range the setup block finds

__global__ void __launch_bounds__(kSetupThreads)
sort_setup(const float *__restrict__ g, int N, SortState *S, int *__restrict__ qdone,
           int qblocks, int with_range) {
    __shared__ int red_lo[kSetupThreads / 32], red_hi[kSetupThreads / 32];
    const int t = threadIdx.x;
    for (int i = t; i <= kSortBuckets; i += kSetupThreads) S->tree_off[i] = S->query_off[i] = 0;
    for (int i = t; i < qblocks; i += kSetupThreads) qdone[i] = 0;
    int lo = 0x7fffffff, hi = (int)0x80000000;
    if (with_range) {
        for (int v = t; v < N; v += kSetupThreads) {
            const float x = g[v];
            if (fabsf(x) <= FLT_MAX) {
                lo = min(lo, fkey(x));
                hi = max(hi, fkey(x));
            }
        }
        lo = __reduce_min_sync(kFull, lo);
        hi = __reduce_max_sync(kFull, hi);
        if ((t & 31) == 0) {
            red_lo[t >> 5] = lo;
            red_hi[t >> 5] = hi;
        }
        __syncthreads();
        if (t == 0)
            for (int w = 1; w < kSetupThreads / 32; ++w) {
                lo = min(lo, red_lo[w]);
                hi = max(hi, red_hi[w]);
            }
    }
    if (t == 0) {
        S->gmin = lo;  // empty finite range: gmin > gmax
        S->gmax = hi;
        S->exact_only = 0;
        S->nonfinite = 0;
        S->maxabs = 0u;
        S->arrive = 0;
    }
}

__global__ void sort_range(const float *__restrict__ g, int N, SortState *S) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    int lo = 0x7fffffff, hi = (int)0x80000000;
    if (v < N) {
        const float x = g[v];
        if (fabsf(x) <= FLT_MAX) lo = hi = fkey(x);
    }
    lo = __reduce_min_sync(kFull, lo);
    hi = __reduce_max_sync(kFull, hi);
    if ((threadIdx.x & 31) == 0 && lo <= hi) {
        atomicMin(&S->gmin, lo);
        atomicMax(&S->gmax, hi);
    }
}

// Warp-aggregated counter update: lanes of a warp with the same bucket b
// (b < 0: no item) add their count once, through the group's first lane, and
// each receives the counter's old value plus its rank in the group (many
// budgets can share one bucket, e.g. every budget above the largest g).
__device__ __forceinline__ int grouped_add(int *counters, int b) {
    const int lane = threadIdx.x & 31;
    const unsigned grp = __match_any_sync(kFull, b);
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (b >= 0 && lane == leader) base = atomicAdd(&counters[b], __popc(grp));
    base = __shfl_sync(kFull, base, leader);
    return base + __popc(grp & ((1u << lane) - 1u));
}

// Bucket counts of the tree's g and of the budgets; the last block to finish
// turns both count arrays into bucket starts.
constexpr int kHistThreads = 256;

__global__ void __launch_bounds__(kHistThreads)
sort_histogram(const float *__restrict__ g, int N, const float *__restrict__ c, int Q,
               SortState *S) {
    __shared__ int s_last;
    __shared__ int part[kHistThreads / 32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float lo, scale;
    g_scale(*S, &lo, &scale);
    grouped_add(S->tree_off + 1, i < N ? sort_bucket(g[i], lo, scale) : -1);
    grouped_add(S->query_off + 1, i < Q ? sort_bucket(c[i], lo, scale) : -1);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&S->arrive, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // inclusive scan of the shifted counts: off[b] becomes the start of
    // bucket b; each thread sums 4 consecutive buckets, then the block scans
    // the 256 sums; the cursors start at the bucket starts
    constexpr int kPer = kSortBuckets / kHistThreads;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    for (int which = 0; which < 2; ++which) {
        int *off = which ? S->query_off : S->tree_off;
        int *cur = which ? S->query_cur : S->tree_cur;
        int v[kPer], own = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            v[k] = __ldcg(off + 1 + kPer * t + k);
            own += v[k];
        }
        int x = own;  // inclusive scan of the thread sums within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) part[w] = x;
        __syncthreads();
        int run = x - own;
        for (int k = 0; k < w; ++k) run += part[k];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            cur[kPer * t + k] = run;  // start of bucket kPer t + k
            run += v[k];
            off[1 + kPer * t + k] = run;
        }
        __syncthreads();  // part is reused
    }
}

// Scatter the tree (all D+1 rows) and the queries into bucket order.
__global__ void sort_scatter(const float *__restrict__ tree, int N, int64_t ld, int dim,
                             const float *__restrict__ queries, const float *__restrict__ budgets,
                             int Q, SortState *S, float *__restrict__ tree_s, int ldt,
                             int *__restrict__ perm, float *__restrict__ q_s,
                             float *__restrict__ c_s, int *__restrict__ qperm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float lo, scale;
    g_scale(*S, &lo, &scale);
    const int bt = i < N ? sort_bucket(tree[(size_t)dim * ld + i], lo, scale) : -1;
    const int pt = grouped_add(S->tree_cur, bt);
    // the TF32 filter's error bound needs every nonzero coordinate in
    // [2^-60, 2^60]; the FP16 filter scales by the largest finite magnitude;
    // NaN and infinities turn either off
    bool out_of_range = false, nonfinite = false;
    unsigned mx = 0u;
    auto check = [&](float v) {
        const float a = fabsf(v);
        out_of_range |= v != 0.f && !(a >= 0x1p-60f && a <= 0x1p60f);
        nonfinite |= !(a <= FLT_MAX);
        if (a <= FLT_MAX) mx = max(mx, __float_as_uint(a));
    };
    if (i < N) {
        // row dim + 1: the FP32 filter's folded squared norm fl(|x|^2) (1 - 4 gamma)
        float n2 = 0.f;
        for (int d = 0; d <= dim; ++d) {
            const float v = tree[(size_t)d * ld + i];
            if (d < dim) {
                check(v);
                n2 = fmaf(v, v, n2);
            }
            tree_s[(size_t)d * ldt + pt] = v;
        }
        tree_s[(size_t)(dim + 1) * ldt + pt] = n2 * (1.f - 4.f * (kF32G * (dim + 2.f)));
        perm[pt] = i;
    }
    const float c = i < Q ? budgets[i] : 0.f;
    const int bq = i < Q ? sort_bucket(c, lo, scale) : -1;
    const int pq = grouped_add(S->query_cur, bq);
    if (i < Q) {
        for (int d = 0; d < dim; ++d) {
            const float v = queries[(size_t)d * Q + i];
            check(v);
            q_s[(size_t)d * Q + pq] = v;
        }
        c_s[pq] = c;
        qperm[pq] = i;
    }
    if (out_of_range) S->exact_only = 1;
    if (nonfinite) S->nonfinite = 1;
    mx = __reduce_max_sync(kFull, mx);
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(&S->maxabs, mx);
}

// Vertices a block of bq consecutive (ordered) queries must scan: up to the
// end of the bucket that holds the largest budget of the block (0 when no
// finite vertex has g below it).  Used by the pair count; a NEAREST call takes
// the cuts from its seeding pass.
__global__ void __launch_bounds__(256) sort_cut(const float *__restrict__ c_s, int Q, int bq,
                                                const SortState *S, int N, int *__restrict__ cut) {
    __shared__ float red[8];
    const int b = blockIdx.x;
    float m = -FLT_MAX;
    for (int i = b * bq + threadIdx.x; i < min(Q, (b + 1) * bq); i += blockDim.x)
        m = fmaxf(m, c_s[i]);  // NaN budgets admit nothing and are ignored here
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) m = fmaxf(m, red[k]);
        m = fmaxf(m, red[0]);
        float lo, scale;
        g_scale(*S, &lo, &scale);
        int n;
        if (S->gmin > S->gmax)
            n = 0;                                 // no finite g at all
        else if (!(m > unkey(S->gmin)))
            n = 0;                                 // no vertex has g < m
        else if (m > unkey(S->gmax))
            n = N;
        else
            n = S->tree_off[sort_bucket(m, lo, scale) + 1];
        cut[b] = n;
    }
}

// Seeding pass, one block per query block: for each (ordered) query, the
// smallest exact squared distance (the filter's own formula) among
// kSeedSamples evenly spaced vertices of the g-ordered tree that are
// admissible for it (+inf when none is), four samples at a time; and the
// block's cut, as sort_cut finds it.
constexpr int kSeedSamples = 64;
template <int DIM>
__global__ void __launch_bounds__(kTcQueries)
nearest_seed(const float *__restrict__ tree_s, int N, int ldt, const float *__restrict__ q_s,
             const float *__restrict__ c_s, int Q, const SortState *S, float *__restrict__ seed,
             int *__restrict__ cut) {
    __shared__ float xs[DIM + 1][kSeedSamples];  // the sample vertices, g in the last row
    __shared__ float red[kTcQueries / 32];
    const int n = min(N, kSeedSamples);
    for (int t = threadIdx.x; t < (DIM + 1) * kSeedSamples; t += blockDim.x) {
        const int d = t / kSeedSamples, k = t % kSeedSamples;
        xs[d][k] = k < n ? tree_s[(size_t)d * ldt + (int)(((int64_t)k * N) / n)] : 0.f;
    }
    __syncthreads();
    const int i = blockIdx.x * kTcQueries + threadIdx.x;
    const float c = i < Q ? c_s[i] : -FLT_MAX;
    if (i < Q) {
        float q[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) q[d] = q_s[(size_t)d * Q + i];
        float best = FLT_MAX * 2.f;
        for (int k = 0; k < n; k += 4) {
            float d2[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int d = 0; d < DIM; ++d)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float a = q[d] - xs[d][k + u];
                    d2[u] = fmaf(a, a, d2[u]);
                }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float g = xs[DIM][k + u];
                if (k + u < n && g < c && g + __fsqrt_rn(d2[u]) < c) best = fminf(best, d2[u]);
            }
        }
        seed[i] = best;
    }
    // the cut: up to the end of the bucket of the block's largest budget
    float m = c;  // NaN budgets admit nothing and are ignored here
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < kTcQueries / 32; ++k) m = fmaxf(m, red[k]);
        float lo, scale;
        g_scale(*S, &lo, &scale);
        int nc;
        if (S->gmin > S->gmax)
            nc = 0;                                 // no finite g at all
        else if (!(m > unkey(S->gmin)))
            nc = 0;                                 // no vertex has g < m
        else if (m > unkey(S->gmax))
            nc = N;
        else
            nc = S->tree_off[sort_bucket(m, lo, scale) + 1];
        cut[blockIdx.x] = nc;
    }
}

// Pairs the budget-ordered pass scans: sum over query blocks of (queries in
// the block) x cut.
__global__ void sort_count_pairs(const int *__restrict__ cut, int qblocks, int Q, int bq,
                                 unsigned long long *out) {
    unsigned long long acc = 0;
    for (int b = threadIdx.x; b < qblocks; b += blockDim.x)
        acc += (unsigned long long)min(bq, Q - b * bq) * (unsigned long long)cut[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// Raises the FP32 filter's dynamic shared-memory limit once per device and
// returns its resident blocks per SM.
template <int DIM>
mrpop_status f32_filter_setup(int dev, int *bps) {
    static std::mutex mu;
    static int done[64] = {};
    static int occ[64] = {};
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64) return set_error(MRPOP_EINVAL, "nearest: device ordinal %d", dev);
    if (!done[dev]) {
        MRPOP_CUDA_TRY(cudaFuncSetAttribute(nearest_f32_kernel<DIM>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)f32_smem_bytes<DIM>()));
        MRPOP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &occ[dev], nearest_f32_kernel<DIM>, kTcThreads, f32_smem_bytes<DIM>()));
        done[dev] = 1;
    }
    *bps = occ[dev];
    return MRPOP_OK;
}

// out_idx null: only count the scanned pairs into *pairs (synchronises).
// filter: MRPOP_NEAREST_FILTER_FP32 (FMA-pipe expansion filter) or
// MRPOP_NEAREST_FILTER_TENSOR (FP16 / TF32 mma.sync expansion filter); both
// decide every survivor exactly, so the indices do not depend on it.
template <int DIM>
mrpop_status nearest_sorted(const float *tree, int N, int64_t ld, const float *queries,
                                const float *budgets, int Q, int64_t *out_idx, cudaStream_t st,
                                int64_t *pairs = nullptr, int filter = MRPOP_NEAREST_FILTER_FP32,
                                int waves = 4) {
    int dev = 0, sms = 1, bps = 1;
    MRPOP_CUDA_TRY(cudaGetDevice(&dev));
    MRPOP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    constexpr bool f16 = DIM + 2 <= 16;  // FP16 tensor filter (K = 16), else TF32
    const bool tensor = filter == MRPOP_NEAREST_FILTER_TENSOR;
    if (!tensor) {
        const mrpop_status fs = f32_filter_setup<DIM>(dev, &bps);
        if (fs != MRPOP_OK) return fs;
    } else if constexpr (f16) {
        MRPOP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, nearest_tc16_kernel<DIM>,
                                                                     kTcThreads, 0));
    } else {
        MRPOP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, nearest_tc_kernel<DIM>,
                                                                     kTcThreads, 0));
    }
    bps = std::max(bps, 1);
    const int bq = kTcQueries;
    const int qblocks = (Q + bq - 1) / bq;
    // about four waves of (query block, tree slice) pieces before the cut
    // removes some: the dynamic block scheduler then evens out the blocks
    // that stop early
    int splits = std::max(1, (std::max(1, waves) * sms * bps + qblocks - 1) / qblocks);
    int chunk = (N + splits - 1) / splits;
    chunk = std::max(kSliceAlign, ((chunk + kSliceAlign - 1) / kSliceAlign) * kSliceAlign);
    splits = std::max(1, (N + chunk - 1) / chunk);
    if (splits > 65535) return set_error(MRPOP_EINVAL, "nearest: tree too large");
    // one stream-ordered arena: sort state, ordered tree and queries,
    // permutations, cuts, partial bests
    auto align = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_state = align(sizeof(SortState));
    // rows of the ordered tree start on 16-byte boundaries (the FP32 filter
    // copies them in 16-byte pieces)
    const int ldt = (N + 3) & ~3;
    const size_t b_tree = align(sizeof(float) * (size_t)(DIM + 2) * ldt);  // + folded norms
    const size_t b_perm = align(sizeof(int) * (size_t)N);
    const size_t b_q = align(sizeof(float) * (size_t)DIM * Q);
    const size_t b_c = align(sizeof(float) * (size_t)Q);
    const size_t b_qp = align(sizeof(int) * (size_t)Q);
    const size_t b_cut = align(sizeof(int) * (size_t)qblocks);
    const size_t b_part = align(sizeof(Best) * (size_t)splits * Q);
    const size_t b_seed = align(sizeof(float) * (size_t)Q);
    const size_t b_qdone = align(sizeof(int) * (size_t)qblocks);
    char *arena = nullptr;
    MRPOP_CUDA_TRY(scratch_alloc((void **)&arena,
                                   b_state + b_tree + b_perm + b_q + b_c + b_qp + b_cut + b_part +
                                       b_seed + b_qdone,
                                   st));
    char *at = arena;
    auto take = [&](size_t b) { char *r = at; at += b; return r; };
    SortState *S = (SortState *)take(b_state);
    float *tree_s = (float *)take(b_tree);
    int *perm = (int *)take(b_perm);
    float *q_s = (float *)take(b_q);
    float *c_s = (float *)take(b_c);
    int *qperm = (int *)take(b_qp);
    int *cut = (int *)take(b_cut);
    Best *partial = (Best *)take(b_part);
    float *seed = (float *)take(b_seed);
    int *qdone = (int *)take(b_qdone);
    const int n_max = std::max(N, Q);
    const float *g = tree + (size_t)DIM * ld;
    // five launches: setup (+ range), histogram (+ scan), scatter, seed (+
    // cut), filter (+ reduce in each query block's last slice)
    const bool setup_range = N <= kSetupRangeMax;
    sort_setup<<<1, kSetupThreads, 0, st>>>(g, N, S, qdone, qblocks, setup_range ? 1 : 0);
    if (!setup_range) sort_range<<<(N + 255) / 256, 256, 0, st>>>(g, N, S);
    sort_histogram<<<(n_max + kHistThreads - 1) / kHistThreads, kHistThreads, 0, st>>>(
        g, N, budgets, Q, S);
    sort_scatter<<<(n_max + 255) / 256, 256, 0, st>>>(tree, N, ld, DIM, queries, budgets, Q, S,
                                                       tree_s, ldt, perm, q_s, c_s, qperm);
    if (!out_idx) {
        sort_cut<<<qblocks, 256, 0, st>>>(c_s, Q, bq, S, N, cut);
        unsigned long long *d_pairs = (unsigned long long *)seed;  // 8 bytes of the arena
        unsigned long long h = 0;
        cudaMemsetAsync(d_pairs, 0, sizeof(unsigned long long), st);
        sort_count_pairs<<<1, 256, 0, st>>>(cut, qblocks, Q, bq, d_pairs);
        cudaMemcpyAsync(&h, d_pairs, sizeof(h), cudaMemcpyDeviceToHost, st);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = cudaGetLastError();
        cudaFreeAsync(arena, st);
        if (e != cudaSuccess) return cuda_error(e, "nearest pair count");
        *pairs = (int64_t)h;
        return MRPOP_OK;
    }
    nearest_seed<DIM><<<qblocks, kTcQueries, 0, st>>>(tree_s, N, ldt, q_s, c_s, Q, S, seed, cut);
    dim3 grid(qblocks, splits);
    const NnFinish fin{qdone, qperm, out_idx};
    if (!tensor)
        nearest_f32_kernel<DIM><<<grid, kTcThreads, f32_smem_bytes<DIM>(), st>>>(
            tree_s, N, ldt, q_s, c_s, Q, chunk, partial, perm, cut, seed, &S->exact_only, fin);
    else if constexpr (f16)
        nearest_tc16_kernel<DIM><<<grid, kTcThreads, 0, st>>>(tree_s, N, ldt, q_s, c_s, Q, chunk,
                                                              partial, perm, cut, seed,
                                                              &S->maxabs, &S->nonfinite, fin);
    else
        nearest_tc_kernel<DIM><<<grid, kTcThreads, 0, st>>>(tree_s, N, ldt, q_s, c_s, Q, chunk, partial,
                                                            perm, cut, seed, &S->exact_only, fin);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(arena, st);
    if (e != cudaSuccess) return cuda_error(e, "nearest (budget-ordered) launch");
    return MRPOP_OK;
}

// NEIGHBORS: a block serves kNbWarps queries, one warp each, and streams the
// tree through shared memory in tiles of kNbTile vertices (SoA rows, loaded
// once for all of the block's queries).  Lanes take 32 consecutive vertices at
// a time in ascending order; ballot + prefix popcount keep the output sorted.
constexpr int kNbWarps = 8;
constexpr int kNbTile = 256;

__global__ void __launch_bounds__(kNbWarps * 32)
neighbors_kernel(const float *__restrict__ tree, int N, int64_t ld, int dim,
                 const float *__restrict__ queries, int Q, float delta, int64_t k_max,
                 int64_t *__restrict__ out_idx, int64_t *__restrict__ out_cnt, int chunk) {
    // blockIdx.y takes vertices [y * chunk, (y + 1) * chunk); with several
    // ranges (gridDim.y > 1) the lists go to per-range slots of out_idx /
    // out_cnt ([q][range]) and neighbors_merge concatenates them in order
    __shared__ float qs[kNbWarps][MRPOP_MAX_LINKS];
    extern __shared__ float tile[];  // [dim][kNbTile]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = blockIdx.x * kNbWarps + warp;
    const bool qok = q < Q;
    for (int d = lane; d < dim; d += 32) qs[warp][d] = qok ? queries[(size_t)d * Q + q] : 0.f;
    const int64_t slot = (int64_t)q * gridDim.y + blockIdx.y;  // this query's range slot
    const int vs = blockIdx.y * chunk, ve = min(N, vs + chunk);
    int64_t count = 0;
    for (int v0 = vs; v0 < ve; v0 += kNbTile) {
        const int nv = min(kNbTile, ve - v0);
        __syncthreads();
        for (int i = threadIdx.x; i < dim * kNbTile; i += blockDim.x) {
            const int d = i / kNbTile, j = i - d * kNbTile;
            tile[i] = j < nv ? __ldg(tree + (size_t)d * ld + v0 + j) : 0.f;
        }
        __syncthreads();
        if (!qok) continue;
        for (int c = 0; c < nv; c += 32) {
            const int v = c + lane;
            bool in = false;
            if (v < nv) {
                float d2 = 0.f;
                for (int d = 0; d < dim; ++d) {
                    const float a = qs[warp][d] - tile[d * kNbTile + v];
                    d2 = fmaf(a, a, d2);
                }
                in = __fsqrt_rn(d2) <= delta;
            }
            const unsigned bal = __ballot_sync(kFull, in);
            if (in) {
                const int64_t pos = count + __popc(bal & ((1u << lane) - 1u));
                if (pos < k_max) out_idx[(size_t)slot * k_max + pos] = v0 + v;
            }
            count += __popc(bal);
        }
    }
    if (!qok) return;
    for (int64_t pos = count + lane; pos < k_max; pos += 32) out_idx[(size_t)slot * k_max + pos] = -1;
    if (lane == 0) out_cnt[slot] = count;
}

// Concatenates each query's per-range lists in range order (ascending vertex
// index), keeping the first k_max, and adds up the counts.
__global__ void neighbors_merge(const int64_t *__restrict__ part_idx,
                                const int64_t *__restrict__ part_cnt, int ranges, int Q,
                                int64_t k_max, int64_t *__restrict__ out_idx,
                                int64_t *__restrict__ out_cnt) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    int64_t total = 0;
    for (int r = 0; r < ranges; ++r) {
        const int64_t slot = (int64_t)q * ranges + r;
        const int64_t c = part_cnt[slot];
        for (int64_t i = 0; i < c && total + i < k_max; ++i)
            out_idx[(size_t)q * k_max + total + i] = part_idx[(size_t)slot * k_max + i];
        total += c;
    }
    for (int64_t pos = total; pos < k_max; ++pos) out_idx[(size_t)q * k_max + pos] = -1;
    out_cnt[q] = total;
}

// C(sigma): segment lengths in FP32, sums in FP64 with a fixed reduction order
// (each block sums a fixed range of segments; one warp adds the block sums in
// block order), so the result is deterministic.
__device__ __forceinline__ double block_sum(double acc, double *red) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    double v = 0.0;
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    }
    return v;  // valid in thread 0
}

__device__ __forceinline__ float segment_length(const float *__restrict__ path, int64_t j, int dim) {
    float s = 0.f;
    for (int d = 0; d < dim; ++d) {
        const float a = path[(j + 1) * dim + d] - path[j * dim + d];
        s = fmaf(a, a, s);
    }
    return __fsqrt_rn(s);
}

__global__ void path_cost_kernel(const float *__restrict__ path, int64_t M, int dim,
                                 int64_t chunk, double *__restrict__ out) {
    __shared__ double red[32];
    const int64_t j0 = (int64_t)blockIdx.x * chunk;
    const int64_t j1 = min(M - 1, j0 + chunk);
    double acc = 0.0;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x)
        acc += (double)segment_length(path, j, dim);
    const double v = block_sum(acc, red);
    if (threadIdx.x == 0) out[blockIdx.x] = v;
}

__global__ void sum_partials_kernel(const double *__restrict__ partial, int n,
                                    double *__restrict__ out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) acc += partial[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
    if (threadIdx.x == 0) *out = acc;
}

}  // namespace

// Tuned-launch cache keys and lookups: the budget-ordered NEAREST's slice
// waves (default 4) and NEIGHBORS's vertex-range target (default 54 warps per
// SM), per (architecture, dimension, log2 of the tree size, log2 of the batch).
static std::string nn_key(const char *kind, int dim, int64_t N, int64_t Q, int filter) {
    return std::string(kind) + " " + tune_arch() + " dim=" + std::to_string(dim) + " N=2^" +
           std::to_string(log2_bucket(N)) + " Q=2^" + std::to_string(log2_bucket(Q)) +
           (filter >= 0 ? " filter=" + std::to_string(filter) : std::string());
}

int nearest_tuned(int dim, int64_t N, int64_t Q, int filter) {
    std::vector<int> v;
    return tune_lookup(nn_key("nearest", dim, N, Q, filter), &v) && !v.empty() && v[0] > 0 ? v[0] : 4;
}

int neighbors_tuned(int dim, int64_t N, int64_t Q) {
    std::vector<int> v;
    return tune_lookup(nn_key("neighbors", dim, N, Q, -1), &v) && !v.empty() && v[0] > 0 ? v[0] : 54;
}

// Times candidates[] (the value passed as the launch knob) with `run`, keeps
// the fastest under key.
template <class Run>
static mrpop_status tune_candidates(const std::string &key, const int *cand, int nc, int reps,
                                    Run run, cudaStream_t st, int32_t *best_out, float *ms_out) {
    cudaEvent_t a, b;
    MRPOP_CUDA_TRY(cudaEventCreate(&a));
    MRPOP_CUDA_TRY(cudaEventCreate(&b));
    float best = INFINITY;
    int bv = 0;
    mrpop_status s = MRPOP_OK;
    for (int i = 0; i < nc && s == MRPOP_OK; ++i) {
        s = run(cand[i]);  // warm
        float tot = 0.f;
        for (int r = 0; r < reps && s == MRPOP_OK; ++r) {
            cudaEventRecord(a, st);
            s = run(cand[i]);
            cudaEventRecord(b, st);
            cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            tot += ms;
        }
        if (s == MRPOP_OK && tot < best) {
            best = tot;
            bv = cand[i];
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (s != MRPOP_OK) return s;
    tune_store(key, {bv});
    if (best_out) *best_out = bv;
    if (ms_out) *ms_out = best / std::max(1, reps);
    return MRPOP_OK;
}

mrpop_status autotune_nearest(const float *tree, int64_t N, int64_t ld, int dim,
                              const float *queries, const float *budgets, int64_t Q,
                              int filter, int64_t *out_idx, int32_t *waves_out, float *ms_out,
                              cudaStream_t st) {
    static const int cand[] = {2, 4, 8};
    return tune_candidates(nn_key("nearest", dim, N, Q, filter), cand, 3, 3,
                           [&](int w) {
                               return launch_nearest(tree, N, ld, dim, queries, budgets, Q,
                                                     out_idx, st, filter, w);
                           },
                           st, waves_out, ms_out);
}

mrpop_status autotune_neighbors(const float *tree, int64_t N, int64_t ld, int dim,
                                const float *queries, int64_t Q, float delta, int64_t k_max,
                                int64_t *out_idx, int64_t *out_cnt, int32_t *target_out,
                                float *ms_out, cudaStream_t st) {
    static const int cand[] = {14, 54, 216};
    return tune_candidates(nn_key("neighbors", dim, N, Q, -1), cand, 3, 3,
                           [&](int t) {
                               return launch_neighbors(tree, N, ld, dim, queries, Q, delta, k_max,
                                                       out_idx, out_cnt, st, t);
                           },
                           st, target_out, ms_out);
}

mrpop_status launch_nearest(const float *tree, int64_t N, int64_t ld, int dim,
                            const float *queries, const float *budgets, int64_t Q,
                            int64_t *out_idx, cudaStream_t st, int filter, int waves) {
    const int n = (int)N, q = (int)Q;
    // Large batches: budget-ordered tree and queries, expansion filter with
    // exact decisions over shared-memory tree tiles.
    if (Q >= 2048 && N > 0) {
        const int w = waves > 0 ? waves : nearest_tuned(dim, N, Q, filter);
        switch (dim) {
            case 3: return nearest_sorted<3>(tree, n, ld, queries, budgets, q, out_idx, st, nullptr, filter, w);
            case 6: return nearest_sorted<6>(tree, n, ld, queries, budgets, q, out_idx, st, nullptr, filter, w);
            case 7: return nearest_sorted<7>(tree, n, ld, queries, budgets, q, out_idx, st, nullptr, filter, w);
            case 14: return nearest_sorted<14>(tree, n, ld, queries, budgets, q, out_idx, st, nullptr, filter, w);
            case 21: return nearest_sorted<21>(tree, n, ld, queries, budgets, q, out_idx, st, nullptr, filter, w);
            case 28: return nearest_sorted<28>(tree, n, ld, queries, budgets, q, out_idx, st, nullptr, filter, w);
            default: break;
        }
    }
    // Small batches (and other dimensions): vertices across lanes, queries
    // broadcast from shared memory, warp-shuffle argmin.
    const int dp = (dim + 3) & ~3;
    switch (dp) {
        case 4: return nearest_dp<4>(tree, n, ld, dim, queries, budgets, q, out_idx, st);
        case 8: return nearest_dp<8>(tree, n, ld, dim, queries, budgets, q, out_idx, st);
        case 12: return nearest_dp<12>(tree, n, ld, dim, queries, budgets, q, out_idx, st);
        case 16: return nearest_dp<16>(tree, n, ld, dim, queries, budgets, q, out_idx, st);
        case 20: return nearest_dp<20>(tree, n, ld, dim, queries, budgets, q, out_idx, st);
        case 24: return nearest_dp<24>(tree, n, ld, dim, queries, budgets, q, out_idx, st);
        case 28: return nearest_dp<28>(tree, n, ld, dim, queries, budgets, q, out_idx, st);
        case 32: return nearest_dp<32>(tree, n, ld, dim, queries, budgets, q, out_idx, st);
        default: break;
    }
    if (dp <= 48) return nearest_dp<48>(tree, n, ld, dim, queries, budgets, q, out_idx, st);
    return nearest_dp<64>(tree, n, ld, dim, queries, budgets, q, out_idx, st);
}

mrpop_status nearest_pairs(const float *tree, int64_t N, int64_t ld, int dim, const float *queries,
                           const float *budgets, int64_t Q, int64_t *pairs, cudaStream_t st) {
    const int n = (int)N, q = (int)Q;
    *pairs = N * Q;  // the small-batch kernels scan every vertex
    if (Q >= 2048 && N > 0) {
        switch (dim) {
            case 3: return nearest_sorted<3>(tree, n, ld, queries, budgets, q, nullptr, st, pairs);
            case 6: return nearest_sorted<6>(tree, n, ld, queries, budgets, q, nullptr, st, pairs);
            case 7: return nearest_sorted<7>(tree, n, ld, queries, budgets, q, nullptr, st, pairs);
            case 14: return nearest_sorted<14>(tree, n, ld, queries, budgets, q, nullptr, st, pairs);
            case 21: return nearest_sorted<21>(tree, n, ld, queries, budgets, q, nullptr, st, pairs);
            case 28: return nearest_sorted<28>(tree, n, ld, queries, budgets, q, nullptr, st, pairs);
            default: break;
        }
    }
    return MRPOP_OK;
}

mrpop_status launch_neighbors(const float *tree, int64_t N, int64_t ld, int dim,
                              const float *queries, int64_t Q, float delta, int64_t k_max,
                              int64_t *out_idx, int64_t *out_cnt, cudaStream_t st,
                              int warps_per_sm) {
    if (warps_per_sm <= 0) warps_per_sm = neighbors_tuned(dim, N, Q);
    const int blocks = (int)((Q + kNbWarps - 1) / kNbWarps);
    const size_t smem = sizeof(float) * (size_t)dim * kNbTile;
    if (smem > 48 * 1024)
        MRPOP_CUDA_TRY(cudaFuncSetAttribute(neighbors_kernel,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // Few queries leave most SMs idle with one warp per query: split the
    // vertices into ranges (at least one tile each) until about warps_per_sm
    // warps per SM run (54 by default: about 8,192 on 152 SMs; tunable).
    int sms = 1, dev = 0;
    MRPOP_CUDA_TRY(cudaGetDevice(&dev));
    MRPOP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t want = std::max<int64_t>(1, (int64_t)sms * std::max(1, warps_per_sm) / std::max<int64_t>(Q, 1));
    const int ranges = (int)std::min<int64_t>(std::min<int64_t>(want, (N + kNbTile - 1) / kNbTile),
                                              std::max<int64_t>(1, 65535));
    if (ranges <= 1 || k_max > 4096) {
        neighbors_kernel<<<blocks, kNbWarps * 32, smem, st>>>(tree, (int)N, ld, dim, queries,
                                                              (int)Q, delta, k_max, out_idx,
                                                              out_cnt, (int)std::max<int64_t>(N, 1));
        MRPOP_CUDA_TRY(cudaGetLastError());
        return MRPOP_OK;
    }
    const int chunk = (int)(((N + ranges - 1) / ranges + kNbTile - 1) / kNbTile * kNbTile);
    const int nr = (int)((N + chunk - 1) / chunk);
    int64_t *part = nullptr;
    const size_t kidx = (size_t)Q * nr * (size_t)std::max<int64_t>(k_max, 1);
    MRPOP_CUDA_TRY(scratch_alloc((void **)&part, sizeof(int64_t) * (kidx + (size_t)Q * nr), st));
    neighbors_kernel<<<dim3(blocks, nr), kNbWarps * 32, smem, st>>>(
        tree, (int)N, ld, dim, queries, (int)Q, delta, k_max, part, part + kidx, chunk);
    neighbors_merge<<<(int)((Q + 127) / 128), 128, 0, st>>>(part, part + kidx, nr, (int)Q, k_max,
                                                           out_idx, out_cnt);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(part, st);
    if (e != cudaSuccess) return cuda_error(e, "neighbors launch");
    return MRPOP_OK;
}

mrpop_status launch_path_cost(const float *path, int64_t M, int dim, double *out,
                              cudaStream_t st) {
    const int threads = 256;
    const int64_t segs = M > 1 ? M - 1 : 0;
    int blocks = (int)std::min<int64_t>(1024, (segs + 4 * threads - 1) / (4 * threads));
    if (blocks <= 1) {
        path_cost_kernel<<<1, threads, 0, st>>>(path, M, dim, segs > 0 ? segs : 1, out);
        MRPOP_CUDA_TRY(cudaGetLastError());
        return MRPOP_OK;
    }
    const int64_t chunk = (segs + blocks - 1) / blocks;
    blocks = (int)((segs + chunk - 1) / chunk);
    double *partial = nullptr;
    MRPOP_CUDA_TRY(scratch_alloc((void **)&partial, sizeof(double) * blocks, st));
    path_cost_kernel<<<blocks, threads, 0, st>>>(path, M, dim, chunk, partial);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        sum_partials_kernel<<<1, 32, 0, st>>>(partial, blocks, out);
        e = cudaGetLastError();
    }
    cudaFreeAsync(partial, st);
    if (e != cudaSuccess) return cuda_error(e, "path cost kernel launch");
    return MRPOP_OK;
}

}  // namespace mrpop

namespace mrpop {

// ---------------------------------------------------------------------------
// Allocation-free NEAREST (mrpop_nearest_noalloc).
//
// mrpop_nearest may take stream-ordered scratch for the partial minima of a
// split tree.  Some callers cannot allocate device memory at query time: a
// real-time replanning loop that must neither stall on the allocator nor risk
// an out-of-memory failure in the middle of a control cycle, or a process whose
// device memory has already been reserved by another framework's caching
// allocator.  For them this variant keeps its partial minima in one fixed
// file-scope device array, g_nearest_noalloc_scratch, which every GPU that
// loads this library holds until the process exits.
//
// Host code cannot use the array's name as a device address (it is a host-side
// stand-in), so every call looks the address up with cudaGetSymbolAddress on
// the current device.  The lookup allocates nothing once the module is loaded
// on that device, which the first call on a device (or any earlier call of
// this library there) does; that first call should therefore come before any
// stream capture.  Not caching the address keeps it right after a device reset
// reloads the module at a new address.  All calls share the array;
// two calls that overlap on the GPU (for example on two streams) race on it.
// Every partial record a call reads was written earlier by the same call, so
// nothing needs clearing between calls.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocRecords = 2 * MRPOP_NEAREST_NOALLOC_MAX_QUERIES;

__device__ __align__(256) Best g_nearest_noalloc_scratch[kNoAllocRecords];

// Device address of the array on the current device (looked up on every call).
mrpop_status noalloc_scratch(Best **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_nearest_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(nearest scratch)");
    *out = static_cast<Best *>(p);
    return MRPOP_OK;
}

template <int DP>
mrpop_status nearest_noalloc_dp(const float *tree, int N, int64_t ld, int dim,
                                const float *queries, const float *budgets, int Q,
                                int64_t *out_idx, Best *scratch, cudaStream_t st) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int groups = (Q + kQB - 1) / kQB;
    const int target = sms * 8;
    int splits = 1;
    if (groups < target && N > 4 * kNNThreads) {
        splits = (target + groups - 1) / groups;
        splits = std::min(splits, (N + 4 * kNNThreads - 1) / (4 * kNNThreads));
    }
    splits = std::max(1, std::min(splits, kNoAllocRecords / Q));
    int chunk = (N + splits - 1) / splits;
    chunk = ((chunk + kNNThreads - 1) / kNNThreads) * kNNThreads;
    if (chunk == 0) chunk = kNNThreads;
    splits = std::max(1, (N + chunk - 1) / chunk);
    dim3 grid(groups, splits);
    nearest_kernel<DP><<<grid, kNNThreads, 0, st>>>(tree, N, ld, dim, queries, budgets, Q, chunk,
                                                    out_idx, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "nearest (no-alloc) kernel launch");
    nearest_reduce_kernel<<<(Q + 255) / 256, 256, 0, st>>>(scratch, splits, Q, out_idx);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "nearest (no-alloc) reduce launch");
    return MRPOP_OK;
}

}  // namespace
}  // namespace mrpop

extern "C" mrpop_status mrpop_nearest_noalloc(const float *tree, int64_t N, int64_t ld,
                                              int32_t dim, const float *queries,
                                              const float *budgets, int64_t Q,
                                              int64_t *out_idx, void *stream) {
    using namespace mrpop;
    if (dim < 1 || dim > MRPOP_MAX_LINKS)
        return set_error(MRPOP_EINVAL, "mrpop_nearest_noalloc: dim=%d outside [1, %d]", dim,
                         MRPOP_MAX_LINKS);
    if (N < 0 || Q < 0 || ld < N || N > (int64_t)INT32_MAX)
        return set_error(MRPOP_EINVAL, "mrpop_nearest_noalloc: bad sizes N=%lld ld=%lld Q=%lld",
                         (long long)N, (long long)ld, (long long)Q);
    if (Q > MRPOP_NEAREST_NOALLOC_MAX_QUERIES)
        return set_error(MRPOP_EINVAL,
                         "mrpop_nearest_noalloc: %lld queries exceed the fixed scratch limit of %d "
                         "(MRPOP_NEAREST_NOALLOC_MAX_QUERIES); split the batch or use mrpop_nearest",
                         (long long)Q, MRPOP_NEAREST_NOALLOC_MAX_QUERIES);
    if (Q == 0) return MRPOP_OK;
    if (!queries || !budgets || !out_idx || (N > 0 && !tree))
        return set_error(MRPOP_EINVAL, "mrpop_nearest_noalloc: NULL buffer");
    Best *scratch = nullptr;
    mrpop_status s = noalloc_scratch(&scratch);
    if (s != MRPOP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int n = (int)N, q = (int)Q;
    switch ((dim + 3) & ~3) {
        case 4: return nearest_noalloc_dp<4>(tree, n, ld, dim, queries, budgets, q, out_idx, scratch, st);
        case 8: return nearest_noalloc_dp<8>(tree, n, ld, dim, queries, budgets, q, out_idx, scratch, st);
        case 12: return nearest_noalloc_dp<12>(tree, n, ld, dim, queries, budgets, q, out_idx, scratch, st);
        case 16: return nearest_noalloc_dp<16>(tree, n, ld, dim, queries, budgets, q, out_idx, scratch, st);
        case 20: return nearest_noalloc_dp<20>(tree, n, ld, dim, queries, budgets, q, out_idx, scratch, st);
        case 24: return nearest_noalloc_dp<24>(tree, n, ld, dim, queries, budgets, q, out_idx, scratch, st);
        case 28: return nearest_noalloc_dp<28>(tree, n, ld, dim, queries, budgets, q, out_idx, scratch, st);
        case 32: return nearest_noalloc_dp<32>(tree, n, ld, dim, queries, budgets, q, out_idx, scratch, st);
        default: break;
    }
    if (((dim + 3) & ~3) <= 48)
        return nearest_noalloc_dp<48>(tree, n, ld, dim, queries, budgets, q, out_idx, scratch, st);
    return nearest_noalloc_dp<64>(tree, n, ld, dim, queries, budgets, q, out_idx, scratch, st);
}

