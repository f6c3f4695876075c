// Batched evaluation of many small, uneven Eq. 1 likelihoods (dense FP64).
//
// Three batched launches prepare every problem at once (K_nu tables of its
// theta, covariance generation, Z into the extra row N); then ONE persistent
// launch factors them all: CTAs take problems from a device queue in the
// order the host gives (largest first, so that the SMs finish together), and
// a CTA (one per SM, 512 threads) runs one problem's whole right-looking
// Cholesky in 64-wide panels -- POTRF of the diagonal block in shared memory,
// TRSM of every row below with the Z row carried along, rank-64 update of the
// trailing lower triangle in 128 x 64 tiles -- and its log-determinant /
// quadratic-form reduction.  No CTA
// waits on another.  Every per-problem quantity (matrix pointer, order, theta
// constants, input pointers) lives in a device descriptor array, so the launch
// sequence of a batch shape (count, orders) is captured once as a CUDA graph
// and replayed with new inputs and theta by refreshing the descriptors.  Each
// problem's result depends only on its own data and a fixed operation order:
// a likelihood is bit-identical alone and inside any batch.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <map>
#include <queue>
#include <mutex>
#include <vector>

#include "geo_internal.cuh"

namespace {

constexpr int PB = 64;   // panel width
constexpr int BT = 256, BR = 128;   // persistent launch: threads per CTA, rows per TRSM chunk / update tile

struct BatchDesc {
    double *A;            // column-major, ld, N columns; row N holds Z' / y'
    long long ld;
    int N, n;
    const double *locs;   // n x 2 (caller order)
    const double *z;      // N
    CovParams cp;
    DevStatus st;         // per-problem status
    DevResults res;
};

// K_nu tables of every problem's theta: block (q, k, problem).
__global__ void __launch_bounds__(32) k_b_cheb_build(BatchDesc *d) {
    __shared__ double hv[GEO_CHEB_N];
    const CovParams &cp = d[blockIdx.z].cp;
    cheb_build_block(cp, const_cast<double *>(cp.tab), blockIdx.x, blockIdx.y, hv);
}

// ---- one persistent launch over the units of every problem ----------------
// A unit is one step of one problem's right-looking Cholesky in 64-wide
// panels: POTRF of the diagonal block (panel c), TRSM of 128 rows below it
// (the Z row included), or one 128 x 64 tile of the rank-64 trailing update
// (the reduction is the unit after the last panel).  The host lays the units
// out in a ticket table, panel-major across the problems (every problem's
// panel-c POTRF, then their TRSM chunks, then their update tiles, then panel
// c + 1 ...), and gives each unit the count of its problem's units that must
// be complete before it starts (all units of the problem's previous phase).
// CTAs take tickets in order; a unit waits (bounded, acquire loads) on its
// problem's done counter, works, and publishes with a release increment.  A
// CTA only waits for units whose tickets were taken earlier by CTAs that are
// running, so the launch cannot deadlock whatever the number of resident CTAs;
// past BWAIT_CYCLES a waiter raises the abort word and records the timeout.
constexpr long long BWAIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz

struct BSmem {
    double S[PB][PB + 1];          // diagonal block, S[col][row]
    union {
        double X[PB][BR + 1];      // TRSM: 128 rows of the panel, X[col][row]
        struct {
            double As[16][BR + 2], Bs[16][PB + 2];   // update: K slices of the two operands
        } u;
        CovParams cp;              // covariance generation: the problem's theta constants
    };
    double red[2][BT / 32];
    int fail, ok;
    int4 unit;
};

__device__ __forceinline__ int b_ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait until *done >= target; false when the launch was aborted (here or elsewhere).
__device__ bool b_wait(const int *done, int target, int *abort_word, int *timeout_word) {
    const long long t0 = clock64();
    for (;;) {
        if (b_ld_acquire(done) >= target) return true;
        if (b_ld_acquire(abort_word)) return false;
        if (clock64() - t0 > BWAIT_CYCLES) {
            atomicExch(abort_word, 1);
            atomicCAS(timeout_word, 0, 7);
            return false;
        }
        __nanosleep(200);
    }
}

__device__ void b_potrf_block(BSmem &sm, double *A, long long ld, int c0, int cb, DevStatus *st) {
    for (int t = threadIdx.x; t < cb * cb; t += BT) {
        const int c = t / cb, r = t % cb;
        sm.S[c][r] = (r >= c) ? __ldcg(A + (long long)(c0 + c) * ld + c0 + r) : 0.0;
    }
    if (threadIdx.x == 0) sm.fail = 0;
    __syncthreads();
    for (int j = 0; j < cb; ++j) {
        if (threadIdx.x == 0) {
            const double v = sm.S[j][j];
            if (!(v > 0.0)) {
                sm.fail = 1;
                st->info = c0 + j + 1;
            } else {
                sm.S[j][j] = sqrt(v);
            }
        }
        __syncthreads();
        if (sm.fail) return;   // uniform
        const double inv = 1.0 / sm.S[j][j];
        for (int r = j + 1 + threadIdx.x; r < cb; r += BT) sm.S[j][r] *= inv;
        __syncthreads();
        const int m = cb - j - 1;
        for (int t = threadIdx.x; t < m * m; t += BT) {
            const int c = j + 1 + t / m, r = j + 1 + t % m;
            if (r >= c) sm.S[c][r] -= sm.S[j][r] * sm.S[j][c];
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < cb * cb; t += BT) {
        const int c = t / cb, r = t % cb;
        if (r >= c) A[(long long)(c0 + c) * ld + c0 + r] = sm.S[c][r];
    }
}

// rows [rbase, rbase + 128) within [c0 + cb, N] (the Z row N included) <- rows L_bb^-T
__device__ void b_trsm_chunk(BSmem &sm, double *A, long long ld, int N, int c0, int cb, int rbase) {
    const int row = threadIdx.x % BR, grp = threadIdx.x / BR;   // 2 groups share the columns
    const int nr = min(BR, N + 1 - rbase);
    for (int t = threadIdx.x; t < cb * cb; t += BT) {
        const int c = t / cb, r = t % cb;
        sm.S[c][r] = (r >= c) ? __ldcg(A + (long long)(c0 + c) * ld + c0 + r) : 0.0;
    }
    for (int t = threadIdx.x; t < cb * BR; t += BT) {
        const int c = t / BR, r = t % BR;
        sm.X[c][r] = (r < nr) ? __ldcg(A + (long long)(c0 + c) * ld + rbase + r) : 0.0;
    }
    __syncthreads();
    for (int c = 0; c < cb; ++c) {
        if (grp == 0) sm.X[c][row] *= 1.0 / sm.S[c][c];
        __syncthreads();
        const double xc = sm.X[c][row];
        for (int k = c + 1 + grp; k < cb; k += BT / BR) sm.X[k][row] -= xc * sm.S[c][k];
        __syncthreads();
    }
    for (int t = threadIdx.x; t < cb * BR; t += BT) {
        const int c = t / BR, r = t % BR;
        if (r < nr) A[(long long)(c0 + c) * ld + rbase + r] = sm.X[c][r];
    }
}

// one 128 x 64 tile (rows t0 + tm.., cols t0 + tn..) of C -= P P', P = cols [c0, c0 + cb)
__device__ void b_update_tile(BSmem &sm, double *A, long long ld, int N, int c0, int cb, int tm, int tn) {
    const int t0 = c0 + cb;
    const int m = N + 1 - t0, n = N - t0;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;   // 16 x 16 threads, 8 x 4 outputs each
    double acc[8][4] = {};
    for (int k0 = 0; k0 < cb; k0 += 16) {
        for (int t = threadIdx.x; t < 16 * BR; t += BT) {
            const int kk = t / BR, r = t % BR;
            sm.u.As[kk][r] = (k0 + kk < cb && tm + r < m) ? __ldcg(A + (long long)(c0 + k0 + kk) * ld + t0 + tm + r) : 0.0;
        }
        for (int t = threadIdx.x; t < 16 * PB; t += BT) {
            const int kk = t / PB, r = t % PB;
            sm.u.Bs[kk][r] = (k0 + kk < cb && tn + r < n) ? __ldcg(A + (long long)(c0 + k0 + kk) * ld + t0 + tn + r) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[8], b[4];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = sm.u.As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = sm.u.Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = tn + tx + 16 * j;
        if (c >= n) continue;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = tm + ty + 16 * i;
            if (r < m && r >= c) {   // the Z row has r > c
                double *pc = A + (long long)(t0 + c) * ld + t0 + r;
                *pc = __ldcg(pc) - acc[i][j];
            }
        }
    }
}

// one 64 x 64 block of location pairs (l in block bl, r in block br <= bl, r <= l) of Eq. 2 into the
// lower triangle; the diagonal blocks also put Z into the extra row N
__device__ void b_covgen_block(BSmem &sm, const BatchDesc &q, int bl, int br) {
    {   // the theta constants into shared memory (every thread reads them per pair)
        const int words = (int)(sizeof(CovParams) / sizeof(int));
        const int *src = reinterpret_cast<const int *>(&q.cp);
        int *dst = reinterpret_cast<int *>(&sm.cp);
        for (int t = threadIdx.x; t < words; t += BT) dst[t] = src[t];
    }
    __syncthreads();
    const CovParams &cp = sm.cp;
    const int p = cp.p, n = q.n;
    const int l = bl * PB + threadIdx.x % PB;
    if (l < n) {
        const double lxv = q.locs[2 * l], lyv = q.locs[2 * l + 1];
        for (int k = threadIdx.x / PB; k < PB; k += BT / PB) {
            const int r = br * PB + k;
            if (r >= n || r > l) continue;
            const double dx = lxv - q.locs[2 * r], dy = lyv - q.locs[2 * r + 1];
            const double x = (l == r) ? 0.0 : sqrt(dx * dx + dy * dy) * cp.inv_a;
            double v[GEO_PMAX_DEV * GEO_PMAX_DEV];
            matern_block(x, cp, v);
            for (int j = 0; j < p; ++j)
                for (int i = 0; i < p; ++i) q.A[(long long)(p * r + j) * q.ld + p * l + i] = v[i * GEO_PMAX_DEV + j];
        }
    }
    if (bl == br)
        for (int t = threadIdx.x; t < p * PB; t += BT) {
            const int k = bl * PB * p + t;
            if (k < q.N) q.A[(long long)k * q.ld + q.N] = q.z[k];
        }
}

__device__ void b_reduce(BSmem &sm, BatchDesc &q) {
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < q.N; k += BT) {
        a += log(__ldcg(q.A + (long long)k * q.ld + k));
        const double v = __ldcg(q.A + (long long)k * q.ld + q.N);
        b += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) sm.red[0][threadIdx.x >> 5] = a, sm.red[1][threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < BT / 32; ++w) ta += sm.red[0][w], tb += sm.red[1][w];
        if (q.st.info) {
            q.res.loglik = q.res.logdet = q.res.quad = nan("");
        } else {
            q.res.logdet = 2.0 * ta;
            q.res.quad = tb;
            q.res.loglik = -0.5 * (double)q.N * log(2.0 * 3.141592653589793) - 0.5 * q.res.logdet - 0.5 * tb;
        }
    }
}

// sync: {ticket, abort, timeout, unused}; done: one counter per problem (all zeroed before the launch).
// units[t] = {problem, kind << 16 | panel, index, target}: kind 0 POTRF, 1 TRSM chunk, 2 update tile
// (index = tile row block * 65536 + tile column block), 3 reduction, 4 covariance block (index = location
// row block * 65536 + location column block); *nunits_p: the unit count.
// Matrix data another CTA wrote is read through L2 (__ldcg), after the acquire of the done counter.
__global__ void __launch_bounds__(BT, 2) k_b_persistent(BatchDesc *d, const int4 *units, const int *nunits_p,
                                                        int *done, int *sync) {
    const int nunits = *nunits_p;
    extern __shared__ __align__(16) uint8_t b_smem_raw[];
    BSmem &sm = *reinterpret_cast<BSmem *>(b_smem_raw);
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(&sync[0], 1);
            sm.unit = t < nunits ? units[t] : make_int4(-1, 0, 0, 0);
            sm.ok = 1;
            if (t < nunits) sm.ok = b_wait(&done[sm.unit.x], sm.unit.w, &sync[1], &sync[2]) ? 1 : 0;
        }
        __syncthreads();
        const int4 u = sm.unit;
        if (u.x < 0 || !sm.ok) return;   // uniform: no more units, or the launch was aborted
        BatchDesc &q = d[u.x];
        const int kind = u.y >> 16, c0 = (u.y & 0xFFFF) * PB;
        // a failed pivot (written before the done counter that this unit waited for) skips the rest
        const bool skip = *(volatile int *)&q.st.info != 0;
        if (kind == 4) {
            b_covgen_block(sm, q, u.z >> 16, u.z & 0xFFFF);
        } else if (!skip || kind == 3) {
            const int cb = min(PB, q.N - c0);
            if (kind == 0)
                b_potrf_block(sm, q.A, q.ld, c0, cb, &q.st);
            else if (kind == 1)
                b_trsm_chunk(sm, q.A, q.ld, q.N, c0, cb, c0 + cb + u.z * BR);
            else if (kind == 2)
                b_update_tile(sm, q.A, q.ld, q.N, c0, cb, (u.z >> 16) * BR, (u.z & 0xFFFF) * PB);
            else
                b_reduce(sm, q);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&done[u.x], 1);
        }
    }
}

}  // namespace

size_t batch_desc_bytes() { return sizeof(BatchDesc); }

// The ticket table.  Per problem the phases run in order -- the covariance
// blocks; for each panel c: POTRF, the TRSM chunks, the update tiles; the
// reduction -- and a unit's
// target is its problem's count of units in earlier phases.  The order of the
// tickets comes from a list-scheduling simulation on `workers` CTAs with
// relative unit costs (update tile 1, TRSM chunk 0.5, POTRF 0.4, covariance
// block 0.3, reduction 0.05): whenever a simulated CTA is free it takes a ready unit of the problem
// with the most work left.  A unit is therefore dispensed only after every
// unit it depends on, and roughly when they complete, so that CTAs rarely
// wait.  Returns the unit count, or minus it when cap (units) is too small.
int batch_units(const int *N, const int *nloc, int count, int workers, void *out_v, size_t cap) {
    int4 *out = (int4 *)out_v;
    struct Phase {
        int kind, c, units;   // kind 0 POTRF, 1 TRSM, 2 update, 3 reduction, 4 covariance blocks
        double cost;          // of one unit
    };
    std::vector<std::vector<Phase>> ph(count);
    std::vector<double> left(count, 0.0);
    size_t total = 0;
    for (int q = 0; q < count; ++q) {
        const int T = (N[q] + PB - 1) / PB;
        const int nbl = (nloc[q] + PB - 1) / PB;
        ph[q].push_back({4, 0, nbl * (nbl + 1) / 2, 0.3});   // covariance blocks (lower triangle of location blocks)
        for (int c = 0; c < T; ++c) {
            const int c0 = c * PB, cb = std::min(PB, N[q] - c0), t0 = c0 + cb;
            ph[q].push_back({0, c, 1, 0.4});
            ph[q].push_back({1, c, (N[q] - t0) / BR + 1, 0.5});   // rows t0 .. N, 128 at a time
            if (t0 < N[q]) {
                const int m = N[q] + 1 - t0, nn = N[q] - t0;
                int tiles = 0;
                for (int tn = 0; tn < nn; tn += PB) tiles += (m - (tn / BR) * BR + BR - 1) / BR;
                ph[q].push_back({2, c, tiles, 1.0});
            }
        }
        ph[q].push_back({3, 0, 1, 0.05});
        for (const Phase &f : ph[q]) left[q] += f.units * f.cost, total += f.units;
    }
    if (!out || cap < total) return -(int)total;
    // simulation state: per problem the current phase, units of it not yet dispensed, running
    std::vector<int> cur(count, 0), undisp(count), running(count, 0), done_before(count, 0);
    for (int q = 0; q < count; ++q) undisp[q] = ph[q][0].units;
    // ready problems by remaining work (max first)
    std::priority_queue<std::pair<double, int>> ready;
    for (int q = 0; q < count; ++q) ready.push({left[q], -q});
    // running units: (finish time, problem), min first
    typedef std::pair<double, int> Ev;
    std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> fin;
    std::vector<double> stale_key(count, -1.0);
    size_t n = 0;
    double now = 0.0;
    int idle = std::max(1, workers);
    while (n < total) {
        // dispense to idle workers while something is ready
        while (idle > 0 && !ready.empty()) {
            const int q = -ready.top().second;
            ready.pop();
            if (undisp[q] == 0) continue;   // stale entry
            const Phase &f = ph[q][cur[q]];
            const int idx = f.units - undisp[q];
            int z = idx;
            if (f.kind == 4) {   // idx -> (location row block, location column block), row by row
                int bl = 0;
                while ((bl + 1) * (bl + 2) / 2 <= idx) ++bl;
                z = bl * 65536 + (idx - bl * (bl + 1) / 2);
            } else if (f.kind == 2) {   // idx -> (tile row block, tile column block), column-major over the triangle
                const int c0 = f.c * PB, cb = std::min(PB, N[q] - c0), t0 = c0 + cb;
                const int m = N[q] + 1 - t0, nn = N[q] - t0;
                int k = idx;
                z = -1;
                for (int tn = 0; tn < nn && z < 0; tn += PB) {
                    const int rows = (m - (tn / BR) * BR + BR - 1) / BR;
                    if (k < rows) z = ((tn / BR) + k) * 65536 + tn / PB;
                    else k -= rows;
                }
            }
            out[n++] = make_int4(q, (f.kind << 16) | f.c, z, done_before[q]);
            --undisp[q];
            ++running[q];
            --idle;
            left[q] -= f.cost;
            fin.push({now + f.cost, q});
            if (undisp[q] > 0) ready.push({left[q], -q});
        }
        if (fin.empty()) break;   // cannot happen: something is running or ready
        // advance to the next completion
        const Ev e = fin.top();
        fin.pop();
        now = e.first;
        const int q = e.second;
        ++idle;
        if (--running[q] == 0 && undisp[q] == 0 && cur[q] + 1 < (int)ph[q].size()) {
            done_before[q] += ph[q][cur[q]].units;   // the phase is complete: the next one is ready
            ++cur[q];
            undisp[q] = ph[q][cur[q]].units;
            ready.push({left[q], -q});
        }
    }
    return (int)n;
}

int batch_workers() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    return 2 * n;   // two CTAs per SM
}

// Builds the descriptors on the host (pinned staging `hdesc`), the launch
// sequence is recorded on `s` (capturable).
struct BatchPlan {
    int count = 0, nmax = 0, Nmax = 0;
};

void batch_fill_desc(void *hdesc_v, int k, double *A, long long ld, int N, int n, const double *locs,
                     const double *z, const CovParams &cp) {
    BatchDesc *h = (BatchDesc *)hdesc_v;
    memset(&h[k], 0, sizeof(BatchDesc));
    h[k].A = A;
    h[k].ld = ld;
    h[k].N = N;
    h[k].n = n;
    h[k].locs = locs;
    h[k].z = z;
    h[k].cp = cp;
}

cudaError_t batch_record(void *ddesc_v, const void *units, const int *nunits, int *counters, int count, int nmax,
                         int Nmax, cudaStream_t s) {
    BatchDesc *d = (BatchDesc *)ddesc_v;
    // counters: sync {ticket, abort, timeout, unused}, then one done counter per problem
    cudaError_t e0 = cudaMemsetAsync(counters, 0, sizeof(int) * (4 + (size_t)count), s);
    if (e0 != cudaSuccess) return e0;
    {
        KScope ks(GEO_K_COVGEN, s);
        k_b_cheb_build<<<dim3(GEO_PMAX_DEV * GEO_PMAX_DEV, GEO_CHEB_NI + 1, count), 32, 0, s>>>(d);
    }
    {
        // covariance generation, factorisation and reduction of every problem in one persistent launch
        KScope ks(GEO_K_GEMM, s);
        cudaError_t e = cudaFuncSetAttribute(k_b_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(BSmem));
        if (e != cudaSuccess) return e;
        k_b_persistent<<<batch_workers(), BT, sizeof(BSmem), s>>>(d, (const int4 *)units, nunits, counters + 4,
                                                                   counters);
    }
    return cudaGetLastError();
}

// Results out of the device descriptors into host arrays (after the stream syncs).
cudaError_t batch_results(const void *ddesc_v, void *hdesc_v, int count, double *loglik, int *info, cudaStream_t s) {
    const BatchDesc *d = (const BatchDesc *)ddesc_v;
    BatchDesc *h = (BatchDesc *)hdesc_v;
    cudaError_t e = cudaMemcpyAsync(h, d, sizeof(BatchDesc) * count, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    for (int k = 0; k < count; ++k) {
        if (loglik) loglik[k] = h[k].res.loglik;
        if (info) info[k] = h[k].st.info;
    }
    return cudaSuccess;
}
