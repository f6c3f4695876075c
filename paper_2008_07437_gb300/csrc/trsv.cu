// Triangular solves with a column-major lower-triangular L (the factor of
// Sigma): forward L x = b and backward L' x = y, the solves of Eq. 1 and of
// the cokriging weights Sigma^-1 Z in Eq. 3.
//
// One launch per solve.  The rows are cut into blocks of 64; CTAs take the
// blocks in solve order from a ticket counter (forward: top to bottom;
// backward: bottom to top).  The CTA holding block I accumulates the products
// with the blocks already solved, waiting on a `done` counter for the ones
// that are not (a block completes only after its predecessor, so one counter
// suffices), then solves its diagonal block with one warp and publishes it.
// A CTA only waits on blocks whose tickets were taken earlier by CTAs that
// are running, so the solve cannot deadlock whatever the number of resident
// CTAs.  Every wait is bounded: past WAIT_CYCLES the CTA raises an abort word
// that makes every other waiter give up too, records the timeout and leaves
// the solve unfinished.  Sums run in a fixed order: the result does not
// depend on timing.  Each pass streams the lower triangle once (HBM-bound).
//
// sync: 4 device ints {ticket, done, abort, unused}, zeroed before each launch.
#include "geo_internal.cuh"

namespace {

constexpr int TB = 64;       // rows per block
constexpr int TT = 256;      // threads per CTA
constexpr long long WAIT_CYCLES = 2000000000LL;   // ~1 s at 2 GHz

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// Wait until done >= target.  Returns done, or -1 when the solve was aborted
// (here or elsewhere).  limit: the wait's clock budget (0 = WAIT_CYCLES).
__device__ int wait_done(int *sync, int target, int *timeout_word, int code, long long limit) {
    const long long t0 = clock64();
    const long long budget = limit > 0 ? limit : WAIT_CYCLES;
    for (;;) {
        const int d = ld_acquire(&sync[1]);
        if (d >= target) return d;
        if (ld_acquire(&sync[2])) return -1;
        if (clock64() - t0 > budget) {
            atomicExch(&sync[2], 1);
            if (timeout_word) atomicCAS(timeout_word, 0, code);
            return -1;
        }
        __nanosleep(100);
    }
}

// Diagonal block Ls[col][row] = L[i0 + row, i0 + col] (row, col < ib) and
// the reciprocals of its diagonal.
__device__ __forceinline__ void load_diag(const double *__restrict__ A, long long ld, int i0, int ib,
                                          double (*Ls)[TB + 1], double *dinv) {
    for (int e = threadIdx.x; e < TB * TB; e += TT) {
        const int c = e / TB, r = e % TB;
        Ls[c][r] = (r < ib && c < ib && r >= c) ? A[(long long)(i0 + c) * ld + i0 + r] : 0.0;
    }
    if (threadIdx.x < ib) dinv[threadIdx.x] = 1.0 / A[(long long)(i0 + threadIdx.x) * ld + i0 + threadIdx.x];
}

__global__ void __launch_bounds__(TT) k_trsv_fwd(const double *__restrict__ A, long long ld, int N, double *x,
                                                 int *sync, int *timeout_word, long long wait_limit) {
    __shared__ double Ls[TB][TB + 1];
    __shared__ double dinv[TB];
    __shared__ double part[TT / TB][TB];
    __shared__ int tick, abort_s;
    const int nblk = (N + TB - 1) / TB;
    const int r = threadIdx.x % TB, g = threadIdx.x / TB;   // row of the block, group of 16 columns
    const int lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) {
            tick = atomicAdd(&sync[0], 1);
            abort_s = 0;
        }
        __syncthreads();
        const int I = tick;
        if (I >= nblk) return;
        const int i0 = I * TB, ib = min(TB, N - i0);
        load_diag(A, ld, i0, ib, Ls, dinv);
        // acc = sum_{J < I} L[i0 + r, J block] x[J block], columns g*16 .. g*16+15 of each block
        double acc = 0.0;
        int seen = 0;
        bool aborted = false;
        for (int J = 0; J < I; ++J) {
            if (J >= seen) {   // warp-uniform
                // every lane waits with its own acquire loads before it reads x
                const int d = __reduce_min_sync(0xffffffffu, wait_done(sync, J + 1, timeout_word, 3, wait_limit));
                if (d < 0) {
                    aborted = true;
                    break;
                }
                seen = d;
            }
            if (r < ib) {
                const double *col = A + (long long)(J * TB + g * 16) * ld + i0 + r;
                const double *xj = x + J * TB + g * 16;
#pragma unroll
                for (int c = 0; c < 16; ++c) acc = fma(col[(long long)c * ld], __ldcg(xj + c), acc);
            }
        }
        if (aborted && lane == 0) atomicExch(&abort_s, 1);
        part[g][r] = acc;
        __syncthreads();
        if (abort_s) return;   // uniform: every thread reads it after the barrier
        if (threadIdx.x < 32) {
            // rows lane and lane + 32 of the block; solve L_II x_I = b_I - part
            const int l = lane;
            double r0 = 0.0, r1 = 0.0;
            if (l < ib) r0 = x[i0 + l] - (part[0][l] + part[1][l] + part[2][l] + part[3][l]);
            if (l + 32 < ib) r1 = x[i0 + l + 32] - (part[0][l + 32] + part[1][l + 32] + part[2][l + 32] + part[3][l + 32]);
            for (int c = 0; c < ib; ++c) {
                const int owner = c & 31;
                double v = 0.0;
                if (l == owner) {
                    if (c < 32) {
                        r0 *= dinv[c];
                        v = r0;
                    } else {
                        r1 *= dinv[c];
                        v = r1;
                    }
                }
                v = __shfl_sync(0xffffffffu, v, owner);
                if (l > c && l < ib) r0 -= Ls[c][l] * v;
                if (l + 32 > c && l + 32 < ib) r1 -= Ls[c][l + 32] * v;
            }
            if (l < ib) x[i0 + l] = r0;
            if (l + 32 < ib) x[i0 + l + 32] = r1;
            __threadfence();
            __syncwarp();
            if (l == 0) st_release(&sync[1], I + 1);
        }
        __syncthreads();   // Ls, part and tick are reused by the next ticket
    }
}

__global__ void __launch_bounds__(TT) k_trsv_bwd(const double *__restrict__ A, long long ld, int N, double *w,
                                                 int *sync, int *timeout_word) {
    __shared__ double Ls[TB][TB + 1];
    __shared__ double dinv[TB];
    __shared__ double part[TB];
    __shared__ int tick, abort_s;
    const int nblk = (N + TB - 1) / TB;
    const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;   // warp: columns 8 warp .. 8 warp + 7
    for (;;) {
        if (threadIdx.x == 0) {
            tick = atomicAdd(&sync[0], 1);
            abort_s = 0;
        }
        __syncthreads();
        const int t = tick;
        if (t >= nblk) return;
        const int I = nblk - 1 - t;
        const int i0 = I * TB, ib = min(TB, N - i0);
        load_diag(A, ld, i0, ib, Ls, dinv);
        // acc[q] = sum_{J > I} sum_{rows k of J} L[k, i0 + 8 warp + q] w[k], lanes over rows
        double acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = 0.0;
        int seen = 0;
        bool aborted = false;
        for (int J = nblk - 1; J > I; --J) {
            const int need = nblk - J;   // tickets 0 .. need-1 done
            if (need > seen) {   // warp-uniform
                // every lane waits with its own acquire loads before it reads w
                const int d = __reduce_min_sync(0xffffffffu, wait_done(sync, need, timeout_word, 4, 0));
                if (d < 0) {
                    aborted = true;
                    break;
                }
                seen = d;
            }
            const int j0 = J * TB, jb = min(TB, N - j0);
            const double w0 = (lane < jb) ? __ldcg(w + j0 + lane) : 0.0;
            const double w1 = (lane + 32 < jb) ? __ldcg(w + j0 + lane + 32) : 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = 8 * warp + q;
                if (c < ib) {
                    const double *col = A + (long long)(i0 + c) * ld + j0;
                    if (lane < jb) acc[q] = fma(col[lane], w0, acc[q]);
                    if (lane + 32 < jb) acc[q] = fma(col[lane + 32], w1, acc[q]);
                }
            }
        }
        if (aborted && lane == 0) atomicExch(&abort_s, 1);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            double v = acc[q];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) part[8 * warp + q] = v;
        }
        __syncthreads();
        if (abort_s) return;
        if (threadIdx.x < 32) {
            // L_II' w_I = y_I - part, from the bottom row up
            const int l = lane;
            double r0 = 0.0, r1 = 0.0;
            if (l < ib) r0 = w[i0 + l] - part[l];
            if (l + 32 < ib) r1 = w[i0 + l + 32] - part[l + 32];
            for (int c = ib - 1; c >= 0; --c) {
                const int owner = c & 31;
                double v = 0.0;
                if (l == owner) {
                    if (c < 32) {
                        r0 *= dinv[c];
                        v = r0;
                    } else {
                        r1 *= dinv[c];
                        v = r1;
                    }
                }
                v = __shfl_sync(0xffffffffu, v, owner);
                // row k < c: r_k -= L[c, k] v, L[c, k] = Ls[k][c]
                if (l < c) r0 -= Ls[l][c] * v;
                if (l + 32 < c) r1 -= Ls[l + 32][c] * v;
            }
            if (l < ib) w[i0 + l] = r0;
            if (l + 32 < ib) w[i0 + l + 32] = r1;
            __threadfence();
            __syncwarp();
            if (l == 0) st_release(&sync[1], t + 1);
        }
        __syncthreads();
    }
}

__global__ void k_copy_strided(const double *__restrict__ in, long long stride, int N, double *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N) out[k] = in[(long long)k * stride];
}

// sync[0] = v (the ticket counter) before a launch
__global__ void k_set_ticket(int *sync, int v) { sync[0] = v; }

int solve_grid(int N) {
    const int nblk = (N + TB - 1) / TB;
    return nblk < 152 * 4 ? nblk : 152 * 4;
}

}  // namespace

cudaError_t forward_solve(const double *A, long long ld, int N, double *x, int *sync, int *timeout_word,
                          cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(sync, 0, 4 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    KScope ks(GEO_K_SOLVE, s, (double)N * N, 8.0 * (double)N * N / 2.0);
    k_trsv_fwd<<<solve_grid(N), TT, 0, s>>>(A, ld, N, x, sync, timeout_word, 0);
    return cudaGetLastError();
}

// The forward solve with its first block withheld: the ticket counter starts
// at 1, so no CTA ever solves block 0 and publishes it, and the CTA of block 1
// waits for a completion that never comes.  With a wait budget of
// wait_limit cycles that wait gives up, raises the abort word (every other
// waiter returns too), records code 3 in *timeout_word and the launch ends.
cudaError_t forward_solve_withheld(const double *A, long long ld, int N, double *x, int *sync, int *timeout_word,
                                   long long wait_limit, cudaStream_t s) {
    if (N <= TB || wait_limit <= 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(sync, 0, 4 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_set_ticket<<<1, 1, 0, s>>>(sync, 1);
    k_trsv_fwd<<<solve_grid(N), TT, 0, s>>>(A, ld, N, x, sync, timeout_word, wait_limit);
    return cudaGetLastError();
}

// w = L^-T y (y strided; w may be y's storage when ystride == 1).
cudaError_t backward_solve(const double *A, long long ld, int N, const double *y, long long ystride, double *w,
                           int *sync, int *timeout_word, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    if (y != w || ystride != 1) {
        KScope ks(GEO_K_AUX, s);
        k_copy_strided<<<(N + 255) / 256, 256, 0, s>>>(y, ystride, N, w);
    }
    cudaError_t e = cudaMemsetAsync(sync, 0, 4 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    KScope ks(GEO_K_SOLVE, s, (double)N * N, 8.0 * (double)N * N / 2.0);
    k_trsv_bwd<<<solve_grid(N), TT, 0, s>>>(A, ld, N, w, sync, timeout_word);
    return cudaGetLastError();
}
