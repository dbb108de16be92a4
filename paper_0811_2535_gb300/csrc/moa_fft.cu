// Plan construction and the C ABI (include/moa_fft.h).
//
// A plan turns the problem statement of Fig. 2.1 (x in C^n, n = 2^t) into a
// short sequence of kernel passes:
//   * 1-D, n <= 4096: one row pass, the whole transform in one tile
//     (the sequential loop of Sec. 3.6 held on chip).
//   * 1-D, n > 4096: dimension lifting n = r*c (Sec. 4.2-4.8, Fig. 4.9):
//     a column pass of r-point transforms with the twiddle w_n^(j2*k1)
//     (block phase), then a row pass of c-point transforms whose store
//     performs the transpose X[k1 + r*k2] (cyclic phase).  Any r*c split
//     is correct (Sec. 4.8); the default is r = 2^floor(t/2).
//     For n = 2^21..2^24 the rows may be lifted once more, c = cA*cB, in
//     one fused launch (three-level lift, lift3.cu), where the autotuner
//     finds it faster.
//   * 2-D / 3-D: the 1-D transform applied along every axis (Omega,
//     Appendix B, Eq. B.6): a row pass on the last axis, column passes on
//     the others; 256^3 arrays in two passes instead, with axis 1 lifted as
//     16 x 16 (plane3d_p1_kernel, then pipe_col_kernel<12,0,3>).
// The autotuner (the paper's script-based search) times the admissible
// choices of a 1-D plan; moa_fft_estimate describes the default plan on the
// host without a GPU.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <cmath>
#include <fstream>
#include <map>
#include <mutex>
#include <string>
#include <sys/stat.h>
#include <unistd.h>
#include <set>
#include <vector>

#include "moa_fft.h"
#include "fft_core.cuh"
#include "batched.h"
#include "internal.h"

using moa::PassDesc;

struct moa_fft_plan_s {
    int dims = 0;
    int64_t n[3] = {0, 0, 0};
    int64_t batch = 0;
    int sign = -1;
    int dtype = 0;
    int64_t total = 0;            // complex elements per exec
    int64_t split_r = 0, split_c = 0;
    std::vector<PassDesc> passes;
    moa::TwiddleSet tw{};
    void *dev_block = nullptr;    // twiddle tables + status word
    float2 *workspace = nullptr;
    size_t workspace_bytes = 0;
    int *d_status = nullptr;
    const float2 *w256 = nullptr;  // two-pass 3-D: w_256^e, e < 256
    // choices an autotuner (or an override) may fix: -1 / 0 = default
    int opt_lr = -1;              // log2 r of a lifted 1-D transform
    int opt_pipe = -1;            // 0: generic kernels only, 1: pipelined strided kernels allowed
    int opt_batch_dlr[17] = {0};  // batched: per log2 length, log2 r offset from floor(log2 n / 2)
    int opt_tile = -1;            // log2 of the tile of the generic passes (10..14)
    int opt_3d2 = -1;             // 3-D 256^3: 1 = two passes, 0 = one pass per axis
    std::string how;              // where the choices came from (defaults, autotuner, its cache)
    int opt_lift3 = -1;           // 1-D: 1 = three-level lift (r = 256, fused second/third pass)
    int opt_sched = -1;           // radix schedule of the generic passes (0..3, see assign_sched)
    bool fault_wait = false;      // MOA_FAULT_WAIT=1 at plan time (tests): short device waits
    bool tma = false;             // tensor-map encoder present: pipelined kernels and the two-pass 3-D plan allowed
    moa::Lift3Launch l3{};
    void *l3_block = nullptr;     // two-level table of w_c, task queue, ticket and unit counters
    // batched plans (moa_fft_plan_batched): one persistent launch
    bool batched = false;
    moa::BatchLaunch bl{};
    void *batch_block = nullptr;  // tasks, offsets, ticket, table pointers
};

namespace {

std::mutex g_plans_mu;
std::set<moa_fft_plan_s *> g_plans;

bool is_live(moa_fft_plan_s *p)
{
    std::lock_guard<std::mutex> lk(g_plans_mu);
    return p && g_plans.count(p) != 0;
}

bool pow2_ge2(int64_t v) { return v >= 2 && (v & (v - 1)) == 0; }

int ilog2(int64_t v)
{
    int l = 0;
    while ((int64_t(1) << l) < v)
        ++l;
    return l;
}

int env_int(const char *name, int fallback)
{
    const char *s = std::getenv(name);
    return (s && *s) ? std::atoi(s) : fallback;
}

// log2 of the tile size in complex elements.  Small tiles let several
// blocks share an SM, so one block's loads overlap another's arithmetic;
// 2^12 (32 KiB) measured best for every pass whose tile can be that small.
// A strided (column) pass needs at least 4 transforms per tile so that every
// row segment it reads or writes is a whole 32-byte sector, and a transposed
// row pass needs 4 rows per tile for the same reason at its store.
// MOA_TILE_LOG2 overrides (10..14) for sweeps.
int tile_log2()
{
    int t = env_int("MOA_TILE_LOG2", 12);
    return t < 10 ? 10 : (t > 14 ? 14 : t);
}

int threads_log2_per_transform(int logN) { return logN < 4 ? 0 : logN - 4; }

int tile_or_default(int tile) { return tile >= 10 && tile <= 14 ? tile : tile_log2(); }

}  // namespace

int moa::pick_logF_col(int logN, int64_t C, int tile)
{
    int lf = tile_or_default(tile) - logN;
    if (lf < 2)
        lf = 2;
    if (lf > moa::max_logF_interleaved(logN))
        lf = moa::max_logF_interleaved(logN);
    const int lf_threads = 10 - threads_log2_per_transform(logN);
    if (lf > lf_threads)
        lf = lf_threads;
    const int lc = ilog2(C);
    if (lf > lc)
        lf = lc;
    return lf < 0 ? 0 : lf;
}

int moa::pick_logF_row(int logN, int64_t O, bool transposed, int tile)
{
    int lf = tile_or_default(tile) - logN;
    if (transposed && lf < 2)
        lf = 2;
    if (transposed && lf > moa::max_logF_interleaved(logN))
        lf = moa::max_logF_interleaved(logN);
    const int lf_threads = 10 - threads_log2_per_transform(logN);
    if (lf > lf_threads)
        lf = lf_threads;
    int lo = 0;
    while ((int64_t(1) << lo) < O)
        ++lo;
    if (lf > lo)
        lf = lo;
    return lf < 0 ? 0 : lf;
}

namespace {

PassDesc row_pass(int logN, int64_t O, int64_t Rt, int src, int dst, int tile)
{
    PassDesc d{};
    d.kind = moa::PASS_ROW;
    d.logN = logN;
    d.O = O;
    d.C = 1;
    d.Rt = Rt;
    d.logF = moa::pick_logF_row(logN, O, Rt > 1, tile);
    d.src = src;
    d.dst = dst;
    d.tw4 = 0;
    return d;
}

PassDesc col_pass(int logN, int64_t O, int64_t C, int tw4, int src, int dst, int tile)
{
    PassDesc d{};
    d.kind = moa::PASS_COL;
    d.logN = logN;
    d.O = O;
    d.C = C;
    d.Rt = 1;
    d.logF = moa::pick_logF_col(logN, C, tile);
    d.src = src;
    d.dst = dst;
    d.tw4 = tw4;
    return d;
}

enum { BUF_IN = 0, BUF_OUT = 1, BUF_WS = 2 };

// Fault injection for host-side tests: MOA_FAULT_ALLOC=1 makes every plan
// allocation fail before cudaMalloc is called.
cudaError_t dev_alloc(void **p, size_t bytes)
{
    if (env_int("MOA_FAULT_ALLOC", 0) == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

void free_plan_memory(moa_fft_plan_s *p)
{
    if (p->l3_block)
        cudaFree(p->l3_block);
    p->l3_block = nullptr;
    if (p->batch_block)
        cudaFree(p->batch_block);
    p->batch_block = nullptr;
    if (p->dev_block)
        cudaFree(p->dev_block);
    if (p->workspace)
        cudaFree(p->workspace);
    p->dev_block = nullptr;
    p->workspace = nullptr;
}

moa_status_t build_passes(moa_fft_plan_s *p)
{
    const int64_t B = p->batch;
    if (p->dtype != MOA_C64) {
        PassDesc d{};
        d.kind = moa::PASS_TC;
        d.logN = ilog2(p->n[0]);
        d.O = B;
        d.C = 1;
        d.Rt = 1;
        d.src = BUF_IN;
        d.dst = BUF_OUT;
        // tcgen05 kernel by default; MOA_TC_KERNEL=sync selects the mma.sync one
        const char *tk = getenv("MOA_TC_KERNEL");
        d.umma = (tk && strcmp(tk, "sync") == 0) ? 0 : 1;
        p->passes.push_back(d);
        return MOA_OK;
    }
    if (p->dims == 1) {
        const int64_t n = p->n[0];
        const int L = ilog2(n);
        if (L <= 12) {
            p->passes.push_back(row_pass(L, B, 1, BUF_IN, BUF_OUT, p->opt_tile));
            return MOA_OK;
        }
        // three-level lift: r = 256 columns pass, then the c = n / 256 point
        // rows as cA x cB in one fused launch (lift3.cu)
        const bool lift3 =
            L >= 21 && L <= 24 && (p->opt_lift3 >= 0 ? p->opt_lift3 == 1 : env_int("MOA_LIFT3", 0) == 1);
        if (lift3) {
            const int lc = L - 8;
            p->split_r = 256;
            p->split_c = int64_t(1) << lc;
            p->passes.push_back(col_pass(8, B, p->split_c, 1, BUF_IN, BUF_WS, p->opt_tile));
            PassDesc d{};
            d.kind = moa::PASS_LIFT3;
            d.logF = (lc + 1) / 2;   // cA
            d.logN = lc / 2;         // cB
            d.O = B * 256;
            d.C = 1;
            d.Rt = 1;
            d.src = BUF_WS;
            d.dst = BUF_OUT;
            p->passes.push_back(d);
            p->workspace_bytes = (size_t)p->total * sizeof(float2);
            return MOA_OK;
        }
        if (L > 24) {
            // n = r*c with r = r1*r2 (Sec. 4.2 applied twice): every factor
            // <= 4096.  Pass 1: r2-point DFTs over the slow index j1s of the
            // rows (stride r1*c) with the twiddle w_r^(j1f*k1s), j1f = the
            // column / c; pass 2: r1-point DFTs over j1f (stride c), the row
            // k1 = k1s + r2*k1f stored in place of the natural r x c layout,
            // with the four-step twiddle w_n^(j2*k1); pass 3: the c-point rows
            // stored transposed at X[k1 + r*k2].
            const int lc = (L + 2) / 3, lr = L - lc;
            const int lr1 = (lr + 1) / 2, lr2 = lr - lr1;
            const int64_t c = int64_t(1) << lc, r1 = int64_t(1) << lr1, r2 = int64_t(1) << lr2;
            p->split_r = int64_t(1) << lr;
            p->split_c = c;
            PassDesc a = col_pass(lr2, B, r1 * c, 1, BUF_IN, BUF_OUT, p->opt_tile);
            a.cdiv = (int)c;
            a.twlog = lr;
            PassDesc b = col_pass(lr1, B * r2, c, 1, BUF_OUT, BUF_WS, p->opt_tile);
            b.Rt = r2;
            p->passes.push_back(a);
            p->passes.push_back(b);
            p->passes.push_back(row_pass(lc, B * p->split_r, p->split_r, BUF_WS, BUF_OUT, p->opt_tile));
            p->workspace_bytes = (size_t)p->total * sizeof(float2);
            return MOA_OK;
        }
        int lr = p->opt_lr >= 0 ? p->opt_lr : env_int("MOA_SPLIT_LOG2R", L / 2);
        if (lr < 1 || lr > 12 || L - lr < 1 || L - lr > 12)
            lr = L / 2;
        const int lc = L - lr;
        p->split_r = int64_t(1) << lr;
        p->split_c = int64_t(1) << lc;
        p->passes.push_back(col_pass(lr, B, p->split_c, 1, BUF_IN, BUF_WS, p->opt_tile));
        p->passes.push_back(row_pass(lc, B * p->split_r, p->split_r, BUF_WS, BUF_OUT, p->opt_tile));
        p->workspace_bytes = (size_t)p->total * sizeof(float2);
        return MOA_OK;
    }
    // 3-D 256^3 in two passes (axis 1 lifted as 16 x 16): axis 2 and the
    // first radix-16 step of axis 1, then the rest of axis 1 and axis 0; 32n
    // bytes instead of the 48n of one pass per axis.  Needs the TMA kernels;
    // MOA_3D_TWO_PASS=0 keeps one pass per axis.
    const int pipe_mode = p->opt_pipe >= 0 ? p->opt_pipe : env_int("MOA_PIPE", 2);
    if (p->dims == 3 && p->n[0] == 256 && p->n[1] == 256 && p->n[2] == 256 && pipe_mode > 0 && p->tma &&
        (p->opt_3d2 >= 0 ? p->opt_3d2 == 1 : env_int("MOA_3D_TWO_PASS", 1) != 0)) {
        PassDesc d1{};
        d1.kind = moa::PASS_PLANE1;
        d1.logN = 8;
        d1.O = B;
        d1.C = 1;
        d1.Rt = 1;
        d1.src = BUF_IN;
        d1.dst = BUF_WS;
        PassDesc d2 = d1;
        d2.kind = moa::PASS_PLANE2;
        d2.logN = 12;
        d2.src = BUF_WS;
        d2.dst = BUF_OUT;
        p->passes.push_back(d1);
        p->passes.push_back(d2);
        p->workspace_bytes = (size_t)p->total * sizeof(float2);
        return MOA_OK;
    }
    const int d = p->dims;
    bool long_axis = false;
    for (int a = 0; a < d; ++a)
        long_axis |= p->n[a] > 4096;
    if (long_axis) {
        // An axis longer than 4096 is lifted L = L1*L2 (element j = js*L1 + jf)
        // inside the array (Sec. 4.2 on one axis, Eq. B.6 on the others): an
        // L2-point pass over js (stride L1*inner) with the twiddle
        // w_L^(jf*ks), jf = the column / inner, then an L1-point pass over jf
        // (stride inner) whose output row ks + L2*kf restores the natural
        // layout.  The passes go through the workspace, the last one into
        // `out`.
        std::vector<PassDesc> ps;
        for (int a = d - 1; a >= 0; --a) {
            int64_t inner = 1, outer = B;
            for (int k = a + 1; k < d; ++k)
                inner *= p->n[k];
            for (int k = 0; k < a; ++k)
                outer *= p->n[k];
            const int l = ilog2(p->n[a]);
            if (l <= 12) {
                ps.push_back(a == d - 1 ? row_pass(l, outer, 1, 0, 0, p->opt_tile)
                                        : col_pass(l, outer, inner, 0, 0, 0, p->opt_tile));
                continue;
            }
            const int l1 = (l + 1) / 2, l2 = l - l1;
            const int64_t L1 = int64_t(1) << l1, L2 = int64_t(1) << l2;
            PassDesc pa = col_pass(l2, outer, L1 * inner, 1, 0, 0, p->opt_tile);
            pa.cdiv = (int)inner;
            pa.twlog = l;
            ps.push_back(pa);
            if (inner == 1) {
                ps.push_back(row_pass(l1, outer * L2, L2, 0, 0, p->opt_tile));
            } else {
                PassDesc pb = col_pass(l1, outer * L2, inner, 0, 0, 0, p->opt_tile);
                pb.Rt = L2;
                ps.push_back(pb);
            }
        }
        // buffers: the last pass writes `out`, the ones before alternate
        // between the workspace and `out`, the first reads `in` (the first
        // pass keeps its own tiles' places, so in == out is allowed)
        int dst = BUF_OUT;
        for (size_t i = ps.size(); i-- > 0;) {
            ps[i].dst = dst;
            dst = dst == BUF_OUT ? BUF_WS : BUF_OUT;
        }
        ps[0].src = BUF_IN;
        for (size_t i = 1; i < ps.size(); ++i)
            ps[i].src = ps[i - 1].dst;
        p->passes = ps;
        p->workspace_bytes = (size_t)p->total * sizeof(float2);
        return MOA_OK;
    }
    // multi-D: last axis as rows, then every other axis as columns, in place
    int src = BUF_IN;
    p->passes.push_back(row_pass(ilog2(p->n[d - 1]), p->total / p->n[d - 1], 1, src, BUF_OUT, p->opt_tile));
    for (int a = d - 2; a >= 0; --a) {
        int64_t inner = 1, outer = B;
        for (int k = a + 1; k < d; ++k)
            inner *= p->n[k];
        for (int k = 0; k < a; ++k)
            outer *= p->n[k];
        p->passes.push_back(col_pass(ilog2(p->n[a]), outer, inner, 0, BUF_OUT, BUF_OUT, p->opt_tile));
    }
    return MOA_OK;
}

// Which strided passes run in the pipelined TMA kernels.  They need the
// tensor-map encoder; without it the plan keeps the generic kernels (same
// results, slower).  MOA_PIPE=0 forces the generic kernels (tests compare
// both paths), MOA_PIPE=1 keeps them but without the blocked workspace.
void assign_pipe(moa_fft_plan_s *p)
{
    const int pipe_mode = p->tma ? (p->opt_pipe >= 0 ? p->opt_pipe : env_int("MOA_PIPE", 2)) : 0;
    for (PassDesc &d : p->passes) {
        // the pipelined kernels take the plain views: no lifted-axis twiddle,
        // no transposed column store
        const bool plain = d.cdiv <= 1 && d.twlog == 0 && (d.kind != moa::PASS_COL || d.Rt <= 1);
        const bool strided4 = plain && d.logN >= 10 && d.logN <= 12 && d.logF == 2 &&
                              (d.kind == moa::PASS_COL ? d.C >= 4 : d.Rt > 1);
        d.pipe = 0;
        d.blk = 0;
        if (strided4 && pipe_mode > 0)
            d.pipe = 1;
    }
    // lifted 1-D with both passes pipelined: the intermediate goes through
    // the workspace as 4 x 4 blocks (whole-block stores in pass 1, whole-block
    // loads in pass 2 instead of 32-byte segments)
    if (pipe_mode >= 2 && p->dims == 1 && p->passes.size() == 2 && p->passes[0].pipe && p->passes[1].pipe &&
        p->passes[0].kind == moa::PASS_COL && p->passes[0].tw4 && p->passes[1].kind == moa::PASS_ROW) {
        p->passes[0].blk = 1;
        p->passes[1].blk = 2;
    }
}

// Radix schedule of every generic row and column pass (the pipelined and
// fused kernels keep their own): 0 = small radix first, 1 = small radix
// last, 2 = radix-8 stages (Sched<logN, V> in fft_core.cuh), 3 = the
// warp-shuffle row kernel for natural-order rows of 128..512 points.  A pass
// for which the chosen schedule does not exist keeps schedule 0.  The
// autotuner's choice, else MOA_SCHED, else 0.
void assign_sched(moa_fft_plan_s *p)
{
    const int want = p->opt_sched >= 0 ? p->opt_sched : env_int("MOA_SCHED", 0);
    for (PassDesc &d : p->passes) {
        d.sched = 0;
        if (d.pipe || (d.kind != moa::PASS_ROW && d.kind != moa::PASS_COL) || want <= 0 || want > 3)
            continue;
        if (!moa::sched_exists(d.logN, want))
            continue;
        // the warp-shuffle kernel: natural-order rows, blocks of 1 to 8 whole warps
        const int threads = moa::pass_threads(d);
        if (want == 3 && (d.kind != moa::PASS_ROW || d.Rt > 1 || threads % 32 != 0 || threads > 256))
            continue;
        d.sched = want;
    }
}

// Device block of the fused second/third pass of a three-level lift: the
// two-level table of w_c (c = cA cB), the ticket and two counters per unit
// (the queue itself is decoded from the ticket), then a ring of four units
// of the intermediate (it stays in L2: rewriting a slot does not send the
// previous unit to DRAM).
moa_status_t build_lift3(moa_fft_plan_s *p, const PassDesc &d)
{
    const int la = d.logF, lb = d.logN, lc = la + lb;
    const int h = (lc + 1) / 2;
    const int64_t rows = d.O;                           // B * r rows of c points
    const int64_t per_unit_rows = int64_t(1) << (12 - lb);
    const int64_t units = rows / per_unit_rows;
    const int per_unit = 1 << la;                       // middle tiles per unit = last tiles per unit
    if (units >= (int64_t(1) << 18) || rows % per_unit_rows)
        return MOA_ERR_UNSUPPORTED;
    const int lag = (int)std::min<int64_t>(2, units);
    const int64_t ntasks = 2 * units * per_unit;
    if (ntasks >= (int64_t(1) << 30))
        return MOA_ERR_UNSUPPORTED;
    const size_t lo_b = ((size_t(1) << h) * sizeof(float2) + 255) & ~size_t(255);
    const size_t hi_b = ((size_t(1) << (lc - h)) * sizeof(float2) + 255) & ~size_t(255);
    const int ring_units = (int)std::min<int64_t>(4, units);
    const size_t ring_b = (size_t)ring_units * (size_t)per_unit_rows * ((size_t)1 << lc) * sizeof(float2);
    const size_t t_b = (((size_t)(1 + 2 * units) * sizeof(int)) + 255) & ~size_t(255);
    const size_t m_b = 2 * sizeof(CUtensorMap);   // the two tensor maps (128-byte aligned at this offset)
    void *blk = nullptr;
    if (dev_alloc(&blk, lo_b + hi_b + t_b + m_b + ring_b) != cudaSuccess)
        return MOA_ERR_ALLOC;
    p->l3_block = blk;
    char *base = static_cast<char *>(blk);
    float2 *lo = reinterpret_cast<float2 *>(base);
    float2 *hi = reinterpret_cast<float2 *>(base + lo_b);
    if (moa::generate_two_level(lo, hi, lc, h, 0) != cudaSuccess)
        return MOA_ERR_CUDA;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MOA_ERR_CUDA;
    moa::Lift3Launch &l = p->l3;
    l.lag = lag;
    l.ticket = reinterpret_cast<int *>(base + lo_b + hi_b);
    CUtensorMap *maps = reinterpret_cast<CUtensorMap *>(base + lo_b + hi_b + t_b);
    l.ring = reinterpret_cast<float2 *>(base + lo_b + hi_b + t_b + m_b);
    l.ring_units = ring_units;
    l.nunits = (int)units;
    l.grid = (int)std::min<int64_t>((int64_t)sms * moa::lift3_blocks_per_sm(), ntasks);
    l.lo = lo;
    l.hi = hi;
    l.h = h;
    l.loga = la;
    l.logb = lb;
    l.logr = 8;
    l.middle_per_unit = per_unit;
    const int fa = 1 << (12 - la), fb = 1 << (12 - lb);
    const int ca = 1 << la, cb = 1 << lb;
    // shared memory: landing buffer (4096 points), exchange buffer, twiddle table
    l.ex_entries = (std::max((ca + ca / 16) * fa, fb * (cb + cb / 16 + 1)) + 15) & ~15;
    l.smem_bytes = (size_t)(4096 + l.ex_entries + 16 * fa) * sizeof(float2) + 64;
    // TMA views: the workspace as [B r cA rows][cB] (middle tiles: cA rows x
    // 4096/cA columns), the ring as [ring rows][cA][cB] (last tiles: the
    // unit's 4096/cB rows at one k2)
    const uint64_t dm[2] = {(uint64_t)cb, (uint64_t)(rows << la)};
    const uint64_t sm_[1] = {(uint64_t)cb * sizeof(float2)};
    const uint32_t bm[2] = {(uint32_t)fa, (uint32_t)ca};
    const uint64_t dl[3] = {(uint64_t)cb, (uint64_t)ca, (uint64_t)(ring_units * per_unit_rows)};
    const uint64_t sl[2] = {(uint64_t)cb * sizeof(float2), ((uint64_t)1 << lc) * sizeof(float2)};
    const uint32_t bl[3] = {(uint32_t)cb, 1, (uint32_t)fb};
    CUtensorMap host_maps[2];
    if (!moa::encode_c64_map(&host_maps[0], p->workspace, 2, dm, sm_, bm) ||
        !moa::encode_c64_map(&host_maps[1], l.ring, 3, dl, sl, bl))
        return MOA_ERR_UNSUPPORTED;
    if (cudaMemcpy(maps, host_maps, sizeof(host_maps), cudaMemcpyHostToDevice) != cudaSuccess)
        return MOA_ERR_CUDA;
    l.map_mid = maps;
    l.map_last = maps + 1;
    return MOA_OK;
}

moa_status_t allocate_and_fill(moa_fft_plan_s *p)
{
    // layout of the device block: status word, stage tables, two-level tables
    bool need_stage[13] = {false};
    for (const PassDesc &d : p->passes) {
        need_stage[d.logN] = true;
        if (d.kind == moa::PASS_LIFT3)
            need_stage[d.logF] = true;
    }
    size_t offs[13] = {0};
    size_t bytes = 256;  // status word
    for (int l = 1; l <= 12; ++l) {
        if (!need_stage[l])
            continue;
        const int ent = moa::stage_table_entries(l);
        if (ent > 0) {
            offs[l] = bytes;
            bytes += ((size_t)ent * sizeof(float2) + 255) & ~size_t(255);
        }
    }
    // tables of the other radix schedules used by the generic passes
    size_t voffs[4][13] = {{0}};
    for (const PassDesc &d : p->passes)
        if (d.sched > 0 && !voffs[d.sched][d.logN]) {
            const int ent = moa::stage_table_entries(d.logN, d.sched);
            if (ent <= 0)
                return MOA_ERR_INVALID_ARG;
            voffs[d.sched][d.logN] = bytes;
            bytes += ((size_t)ent * sizeof(float2) + 255) & ~size_t(255);
        }
    size_t lo_off = 0, hi_off = 0;
    int logn = 0, h = 0;
    if (p->split_r > 0) {
        logn = ilog2(p->total / p->batch);
        h = (logn + 1) / 2;
        lo_off = bytes;
        bytes += ((size_t(1) << h) * sizeof(float2) + 255) & ~size_t(255);
        hi_off = bytes;
        bytes += ((size_t(1) << (logn - h)) * sizeof(float2) + 255) & ~size_t(255);
    }
    // further two-level tables w_M (lifted axes), one per order M
    size_t x_lo_off[32] = {0}, x_hi_off[32] = {0};
    for (const PassDesc &d : p->passes)
        if (d.twlog > 0 && d.twlog < 32 && !x_lo_off[d.twlog]) {
            const int xh = (d.twlog + 1) / 2;
            x_lo_off[d.twlog] = bytes;
            bytes += ((size_t(1) << xh) * sizeof(float2) + 255) & ~size_t(255);
            x_hi_off[d.twlog] = bytes;
            bytes += ((size_t(1) << (d.twlog - xh)) * sizeof(float2) + 255) & ~size_t(255);
        }
    size_t w256_off = 0;
    for (const PassDesc &d : p->passes)
        if (d.kind == moa::PASS_PLANE1 && !w256_off) {
            w256_off = bytes;
            bytes += (257 * sizeof(float2) + 255) & ~size_t(255);
        }
    size_t tc_off = 0;
    if (p->dtype != MOA_C64) {
        tc_off = bytes;
        bytes += ((size_t)moa::tc_table_entries(p->passes[0].logN) * sizeof(float2) + 255) & ~size_t(255);
    }
    void *blk = nullptr;
    if (dev_alloc(&blk, bytes) != cudaSuccess)
        return MOA_ERR_ALLOC;
    p->dev_block = blk;
    if (p->workspace_bytes) {
        void *ws = nullptr;
        if (dev_alloc(&ws, p->workspace_bytes) != cudaSuccess)
            return MOA_ERR_ALLOC;
        p->workspace = static_cast<float2 *>(ws);
    }
    char *base = static_cast<char *>(blk);
    p->d_status = reinterpret_cast<int *>(base);
    if (cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess)
        return MOA_ERR_CUDA;
    if (moa::prepare_kernels() != cudaSuccess)
        return MOA_ERR_CUDA;
    if (moa::prepare_pipe_kernels() != cudaSuccess)
        return MOA_ERR_CUDA;
    for (int l = 1; l <= 12; ++l) {
        p->tw.stage[l] = nullptr;
        if (offs[l]) {
            p->tw.stage[l] = reinterpret_cast<float2 *>(base + offs[l]);
            if (moa::generate_stage_table(const_cast<float2 *>(p->tw.stage[l]), l, 0) != cudaSuccess)
                return MOA_ERR_CUDA;
        }
        for (int v = 0; v < 4; ++v) {
            p->tw.vstage[v][l] = nullptr;
            if (v > 0 && voffs[v][l]) {
                float2 *t = reinterpret_cast<float2 *>(base + voffs[v][l]);
                if (moa::generate_stage_table(t, l, 0, v) != cudaSuccess)
                    return MOA_ERR_CUDA;
                p->tw.vstage[v][l] = t;
            }
        }
    }
    if (tc_off) {
        float2 *t = reinterpret_cast<float2 *>(base + tc_off);
        const int L = p->passes[0].logN;
        if (moa::generate_full_stage(t, int64_t(1) << L, int64_t(1) << (L - 4), 0) != cudaSuccess)
            return MOA_ERR_CUDA;
        if (L == 12 && moa::generate_full_stage(t + 16 * 256, 256, 16, 0) != cudaSuccess)
            return MOA_ERR_CUDA;
        p->tw.tc = t;
    }
    if (w256_off) {
        float2 *t = reinterpret_cast<float2 *>(base + w256_off);
        if (moa::generate_two_level(t, t + 256, 8, 8, 0) != cudaSuccess)   // t[e] = w_256^e
            return MOA_ERR_CUDA;
        p->w256 = t;
    }
    if (p->split_r > 0) {
        float2 *lo = reinterpret_cast<float2 *>(base + lo_off);
        float2 *hi = reinterpret_cast<float2 *>(base + hi_off);
        if (moa::generate_two_level(lo, hi, logn, h, 0) != cudaSuccess)
            return MOA_ERR_CUDA;
        p->tw.lo = lo;
        p->tw.hi = hi;
        p->tw.h = h;
    }
    for (int l = 1; l < 32; ++l) {
        p->tw.xlo[l] = p->tw.xhi[l] = nullptr;
        p->tw.xh[l] = 0;
        if (!x_lo_off[l])
            continue;
        const int xh = (l + 1) / 2;
        float2 *lo = reinterpret_cast<float2 *>(base + x_lo_off[l]);
        float2 *hi = reinterpret_cast<float2 *>(base + x_hi_off[l]);
        if (moa::generate_two_level(lo, hi, l, xh, 0) != cudaSuccess)
            return MOA_ERR_CUDA;
        p->tw.xlo[l] = lo;
        p->tw.xhi[l] = hi;
        p->tw.xh[l] = xh;
    }
    for (const PassDesc &d : p->passes)
        if (d.kind == moa::PASS_LIFT3) {
            const moa_status_t st = build_lift3(p, d);
            if (st != MOA_OK)
                return st;
        }
    if (cudaDeviceSynchronize() != cudaSuccess)
        return MOA_ERR_CUDA;
    return MOA_OK;
}

moa_status_t check_io(const void *in, const void *out)
{
    if (!in || !out || (reinterpret_cast<uintptr_t>(in) & 7) || (reinterpret_cast<uintptr_t>(out) & 7))
        return MOA_ERR_INVALID_ARG;
    return MOA_OK;
}


// ---------------------------------------------------------------------------
// Batched plans: transforms of uneven lengths in one persistent launch.

// Split of a large transform (2^13..2^16 points) handled inside one block:
// both factors in [16, 1024] (so every tile holds at least four transforms);
// default r = 2^floor(log n / 2), MOA_BATCH_LOG2R overrides within range.
int batched_logr(int logn, int dlr)
{
    const int lo = std::max(4, logn - 10), hi = std::min(10, logn - 4);
    const int dflt = std::min(std::max(logn / 2 + dlr, lo), hi);
    int lr = env_int("MOA_BATCH_LOG2R", dflt);
    if (lr < lo || lr > hi)
        lr = dflt;
    return lr;
}

// The host part of a batched plan: the transforms grouped by length, longest
// first (offs_sorted: their offsets in that order), and the work queue of
// small tasks and large-transform tiles.  `resident` is the number of
// persistent blocks that run at once (SMs x blocks per SM).
struct BatchQueue {
    std::vector<int64_t> offs_sorted;
    std::vector<moa::BatchTask> queue;
    bool need_stage[13] = {false};
    bool need_lift[17] = {false};
    bool has_large = false;
};

void build_queue(const int64_t *lengths, int64_t count, const int *dlr, int64_t resident, BatchQueue &bq)
{
    std::vector<int64_t> offset(count);
    int64_t total = 0;
    for (int64_t i = 0; i < count; ++i) {
        offset[i] = total;
        total += lengths[i];
    }
    std::vector<int64_t> &offs_sorted = bq.offs_sorted;
    bool *need_stage = bq.need_stage;
    bool *need_lift = bq.need_lift;
    // group by length, longest first
    offs_sorted.reserve(count);
    std::vector<moa::BatchTask> small;
    std::vector<double> small_cost;
    std::vector<int> large;   // positions in offs_sorted of the large transforms, longest first
    std::vector<int8_t> large_logn;
    for (int logn = 16; logn >= 1; --logn) {
        std::vector<int64_t> group;
        for (int64_t i = 0; i < count; ++i)
            if (ilog2(lengths[i]) == logn)
                group.push_back(offset[i]);
        if (group.empty())
            continue;
        const int first = (int)offs_sorted.size();
        offs_sorted.insert(offs_sorted.end(), group.begin(), group.end());
        if (logn >= 13) {
            const int lr = batched_logr(logn, dlr[logn]);
            need_stage[lr] = need_stage[logn - lr] = true;
            need_lift[logn] = true;
            for (size_t k = 0; k < group.size(); ++k) {
                large.push_back(first + (int)k);
                large_logn.push_back((int8_t)logn);
            }
        } else {
            need_stage[logn] = true;
            const int fmax = logn <= 4 ? 256 : (4096 >> logn);
            for (size_t k = 0; k < group.size(); k += fmax) {
                const int cnt = (int)std::min<size_t>(fmax, group.size() - k);
                small.push_back(moa::BatchTask{first + (int)k, (int16_t)cnt, 0, (int8_t)logn, 0, 0, 0});
                small_cost.push_back((double)cnt * (double)(int64_t(1) << logn));
            }
        }
    }
    // Queue: the column tiles of the large transforms in order; each
    // transform's row tiles follow its last column tile about one wave of
    // blocks later (so its workspace is still in L2 when read back and the
    // row tiles rarely wait); then the small tasks, longest first.
    std::vector<moa::BatchTask> &queue = bq.queue;
    {
        struct Pending {
            size_t idx;
            int64_t ready_at;
        };
        std::vector<Pending> pending;
        size_t next_pending = 0;
        int64_t emitted_cols = 0;
        auto emit_rows = [&](size_t li) {
            const int logn = large_logn[li], lr = batched_logr(logn, dlr[logn]);
            for (int g = 0; g < (1 << (logn - 12)); ++g)
                queue.push_back(moa::BatchTask{large[li], 1, (int16_t)g, (int8_t)logn, (int8_t)lr, 2, 0});
        };
        for (size_t li = 0; li < large.size(); ++li) {
            const int logn = large_logn[li], lr = batched_logr(logn, dlr[logn]);
            for (int g = 0; g < (1 << (logn - 12)); ++g) {
                queue.push_back(moa::BatchTask{large[li], 1, (int16_t)g, (int8_t)logn, (int8_t)lr, 1, 0});
                ++emitted_cols;
                while (next_pending < pending.size() && pending[next_pending].ready_at <= emitted_cols)
                    emit_rows(pending[next_pending++].idx);
            }
            pending.push_back(Pending{li, emitted_cols + resident});
        }
        while (next_pending < pending.size())
            emit_rows(pending[next_pending++].idx);
        std::vector<size_t> order(small.size());
        for (size_t i = 0; i < order.size(); ++i)
            order[i] = i;
        std::stable_sort(order.begin(), order.end(),
                         [&](size_t a, size_t b) { return small_cost[a] > small_cost[b]; });
        for (size_t i : order)
            queue.push_back(small[i]);
    }

    bq.has_large = !large.empty();
}

moa_status_t build_batched(moa_fft_plan_s *p, const int64_t *lengths, int64_t count)
{
    int64_t total = 0;
    for (int64_t i = 0; i < count; ++i)
        total += lengths[i];
    p->total = total;
    p->batch = 1;
    p->dims = 1;
    p->batched = true;

    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MOA_ERR_CUDA;
    const int64_t resident = (int64_t)sms * moa::batched_blocks_per_sm();

    BatchQueue bq;
    build_queue(lengths, count, p->opt_batch_dlr, resident, bq);
    const std::vector<int64_t> &offs_sorted = bq.offs_sorted;
    const std::vector<moa::BatchTask> &queue = bq.queue;
    const bool *need_stage = bq.need_stage;
    const bool *need_lift = bq.need_lift;

    // device block: status | tasks | offsets | ticket | tables struct | stage tables | two-level tables
    auto align = [](size_t v) { return (v + 255) & ~size_t(255); };
    size_t bytes = 256;
    const size_t tasks_off = bytes;
    bytes = align(bytes + queue.size() * sizeof(moa::BatchTask));
    const size_t offs_off = bytes;
    bytes = align(bytes + offs_sorted.size() * sizeof(int64_t));
    const size_t ticket_off = bytes;   // ticket, then one completion counter per transform
    bytes = align(bytes + sizeof(int) * (size_t)(1 + count));
    const size_t tables_off = bytes;
    bytes = align(bytes + sizeof(moa::BatchTables));
    size_t stage_off[13] = {0}, lo_off[17] = {0}, hi_off[17] = {0};
    for (int l = 1; l <= 12; ++l)
        if (need_stage[l] && moa::stage_table_entries(l) > 0) {
            stage_off[l] = bytes;
            bytes = align(bytes + (size_t)moa::stage_table_entries(l) * sizeof(float2));
        }
    for (int l = 13; l <= 16; ++l)
        if (need_lift[l]) {
            const int h = (l + 1) / 2;
            lo_off[l] = bytes;
            bytes = align(bytes + (size_t(1) << h) * sizeof(float2));
            hi_off[l] = bytes;
            bytes = align(bytes + (size_t(1) << (l - h)) * sizeof(float2));
        }
    void *blk = nullptr;
    if (dev_alloc(&blk, bytes) != cudaSuccess)
        return MOA_ERR_ALLOC;
    p->batch_block = blk;
    if (bq.has_large) {
        void *ws = nullptr;
        p->workspace_bytes = (size_t)total * sizeof(float2);
        if (dev_alloc(&ws, p->workspace_bytes) != cudaSuccess)
            return MOA_ERR_ALLOC;
        p->workspace = static_cast<float2 *>(ws);
    }
    char *base = static_cast<char *>(blk);
    p->d_status = reinterpret_cast<int *>(base);
    if (moa::prepare_kernels() != cudaSuccess)
        return MOA_ERR_CUDA;
    moa::BatchTables tb{};
    for (int l = 1; l <= 12; ++l)
        if (stage_off[l]) {
            float2 *t = reinterpret_cast<float2 *>(base + stage_off[l]);
            if (moa::generate_stage_table(t, l, 0) != cudaSuccess)
                return MOA_ERR_CUDA;
            tb.stage[l] = t;
        }
    for (int l = 13; l <= 16; ++l)
        if (need_lift[l]) {
            float2 *lo = reinterpret_cast<float2 *>(base + lo_off[l]);
            float2 *hi = reinterpret_cast<float2 *>(base + hi_off[l]);
            if (moa::generate_two_level(lo, hi, l, (l + 1) / 2, 0) != cudaSuccess)
                return MOA_ERR_CUDA;
            tb.lo[l] = lo;
            tb.hi[l] = hi;
            tb.h[l] = (l + 1) / 2;
        }
    if (cudaMemset(base, 0, 256) != cudaSuccess ||
        cudaMemcpy(base + tasks_off, queue.data(), queue.size() * sizeof(moa::BatchTask), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(base + offs_off, offs_sorted.data(), offs_sorted.size() * sizeof(int64_t),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(base + tables_off, &tb, sizeof(tb), cudaMemcpyHostToDevice) != cudaSuccess)
        return MOA_ERR_CUDA;
    p->bl.tasks = reinterpret_cast<const moa::BatchTask *>(base + tasks_off);
    p->bl.ntasks = (int)queue.size();
    p->bl.ticket = reinterpret_cast<int *>(base + ticket_off);
    p->bl.ncounters = (int)count;
    p->bl.offs = reinterpret_cast<const int64_t *>(base + offs_off);
    p->bl.ws = p->workspace;
    p->bl.tables = reinterpret_cast<const moa::BatchTables *>(base + tables_off);
    const int64_t grid = std::min<int64_t>(resident, (int64_t)queue.size());
    p->bl.grid = (unsigned)std::max<int64_t>(grid, 1);
    // a row tile polls its counter (64 ns sleep each) far beyond the few
    // microseconds a column tile takes; MOA_FAULT_WAIT=1 (tests) makes every
    // row-tile wait unreachable and short, so the timeout path runs
    const bool fault_wait = env_int("MOA_FAULT_WAIT", 0) == 1;
    p->bl.max_polls = fault_wait ? 256 : (1 << 22);
    p->bl.wait_extra = fault_wait ? 1 : 0;
    if (cudaDeviceSynchronize() != cudaSuccess)
        return MOA_ERR_CUDA;
    return MOA_OK;
}

moa_status_t run_pass(moa_fft_plan_s *p, size_t i, const void *in, void *out, cudaStream_t s, int sign)
{
    if (p->batched) {
        const int flags = sign > 0 ? (moa::FLAG_CONJ_IN | moa::FLAG_CONJ_OUT) : 0;
        return moa::launch_batched(p->bl, static_cast<const float2 *>(in), static_cast<float2 *>(out), flags, s,
                                   p->d_status) == cudaSuccess
                   ? MOA_OK
                   : MOA_ERR_CUDA;
    }
    PassDesc d = p->passes[i];
    const size_t np = p->passes.size();
    // The blocked intermediate needs pass 1 on the TMA kernel, which needs a
    // 16-byte aligned input; with an input that is only 8-byte aligned this
    // exec runs both passes in the natural layout instead (generic column
    // pass, then the transposed row pass).
    if (p->passes[0].blk == 1 && (reinterpret_cast<uintptr_t>(in) & 15) != 0)
        d.blk = 0;
    auto buf = [&](int id) -> float2 * {
        return id == BUF_IN ? const_cast<float2 *>(static_cast<const float2 *>(in))
                            : (id == BUF_OUT ? static_cast<float2 *>(out) : p->workspace);
    };
    // sign +1 is conj(F_-(conj x)): conjugate on the first load and last store
    int flags = 0;
    if (sign > 0) {
        if (i == 0)
            flags |= moa::FLAG_CONJ_IN;
        if (i + 1 == np)
            flags |= moa::FLAG_CONJ_OUT;
    }
    // programmatic dependent launch (MOA_PDL=0: plain stream order): every
    // pass after the first, and a first pass that is a pipelined kernel (it
    // lands its first tile as soon as the kernel before it completes).  A
    // generic first pass launches in plain order: measured on the GB300, it
    // ran slower when its blocks were placed early behind a pipelined kernel.
    if (env_int("MOA_PDL", 1) && (i > 0 || d.pipe))
        flags |= moa::FLAG_PDL;
    // fault injection (MOA_FAULT_WAIT=1 at plan time): the pipelined kernels
    // give up on a tile load that has not landed at its first test
    if (p->fault_wait)
        flags |= moa::FLAG_SHORT_WAIT;
    if (d.kind == moa::PASS_LIFT3)   // reads the workspace through the tensor map made at plan time
        return moa::launch_lift3(p->l3, buf(d.dst), p->tw.stage[d.logF], p->tw.stage[d.logN], flags, s,
                                 p->d_status) == cudaSuccess
                   ? MOA_OK
                   : MOA_ERR_CUDA;
    if (d.kind == moa::PASS_PLANE1)
        return moa::launch_plane1(d, buf(d.src), buf(d.dst), p->tw, p->w256, flags, s) == cudaSuccess ? MOA_OK
                                                                                                       : MOA_ERR_CUDA;
    if (d.kind == moa::PASS_PLANE2)
        return moa::launch_pipe_plane2(d, buf(d.src), buf(d.dst), p->tw, flags, s, p->d_status) == cudaSuccess
                   ? MOA_OK
                   : MOA_ERR_CUDA;
    if (d.kind == moa::PASS_TC) {
        const bool bf16 = p->dtype == MOA_C64_TC_BF16;
        const cudaError_t e = d.umma ? moa::launch_umma_pass(d, bf16, buf(d.src), buf(d.dst), p->tw.tc, flags, s,
                                                             p->d_status)
                                     : moa::launch_tc_pass(d, bf16, buf(d.src), buf(d.dst), p->tw.tc, flags, s);
        return e == cudaSuccess ? MOA_OK : MOA_ERR_CUDA;
    }
    if (moa::launch_pass(d, buf(d.src), buf(d.dst), p->tw, flags, s, p->d_status) != cudaSuccess)
        return MOA_ERR_CUDA;
    return MOA_OK;
}

moa_status_t run_unchecked(moa_fft_plan_s *p, const void *in, void *out, cudaStream_t s, int sign)
{
    const size_t np = p->batched ? 1 : p->passes.size();
    for (size_t i = 0; i < np; ++i) {
        const moa_status_t st = run_pass(p, i, in, out, s, sign);
        if (st != MOA_OK)
            return st;
    }
    return MOA_OK;
}


// ---------------------------------------------------------------------------
// Autotuner.  The paper leaves the blocking (breakpoint) to the user and
// proposes a script-based search over alternatives (Sec. 4.8, Sec. 8); the
// plan does that search itself.  For a lifted 1-D transform it times every
// valid r x c split with and without the pipelined strided kernels; for a
// batched plan, three split policies for its large transforms.  Results are
// kept per process and in a small text cache (MOA_TUNE_CACHE, default
// $HOME/.cache/moafft/tune.txt) keyed by GPU name.  MOA_AUTOTUNE=0 keeps
// the defaults; an explicit MOA_SPLIT_LOG2R / MOA_PIPE / MOA_BATCH_LOG2R
// override also skips the search.

std::mutex g_tune_mu;
std::map<std::string, std::string> g_tune;
bool g_tune_loaded = false;

std::string tune_path()
{
    const char *e = std::getenv("MOA_TUNE_CACHE");
    if (e && *e)
        return e;
    const char *h = std::getenv("HOME");
    return std::string(h && *h ? h : "/tmp") + "/.cache/moafft/tune.txt";
}

void tune_load_locked()
{
    if (g_tune_loaded)
        return;
    g_tune_loaded = true;
    std::ifstream f(tune_path());
    std::string key, value;
    while (f >> key && std::getline(f, value)) {
        const size_t b = value.find_first_not_of(' ');
        g_tune[key] = b == std::string::npos ? "" : value.substr(b);
    }
}

bool tune_get(const std::string &key, std::string &value)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(key);
    if (it == g_tune.end())
        return false;
    value = it->second;
    return true;
}

void tune_put(const std::string &key, const std::string &value)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    g_tune[key] = value;
    const std::string path = tune_path();
    const size_t slash = path.rfind('/');
    if (slash != std::string::npos) {   // create up to two missing directory levels
        const std::string dir = path.substr(0, slash);
        const size_t s2 = dir.rfind('/');
        if (s2 != std::string::npos)
            mkdir(dir.substr(0, s2).c_str(), 0755);
        mkdir(dir.c_str(), 0755);
    }
    const std::string tmp = path + ".tmp" + std::to_string((long)getpid());
    {
        std::ofstream f(tmp);
        if (!f)
            return;
        for (const auto &kv : g_tune)
            f << kv.first << ' ' << kv.second << '\n';
    }
    std::rename(tmp.c_str(), path.c_str());
}

std::string device_tag()
{
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return "unknown";
    std::string t = prop.name;
    for (char &ch : t)
        if (ch == ' ')
            ch = '_';
    return t;
}

// Mean time of one exec on scratch buffers (zeros); +inf on any failure.
float time_exec(moa_fft_plan_s *p)
{
    const size_t bytes = (size_t)p->total * sizeof(float2);
    void *a = nullptr, *b = nullptr;
    if (dev_alloc(&a, bytes) != cudaSuccess)
        return INFINITY;
    if (dev_alloc(&b, bytes) != cudaSuccess) {
        cudaFree(a);
        return INFINITY;
    }
    float ms = INFINITY;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMemset(a, 0, bytes) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess) {
        bool ok = true;
        for (int i = 0; i < 2 && ok; ++i)
            ok = run_unchecked(p, a, b, 0, -1) == MOA_OK;
        const int reps = 5;
        ok = ok && cudaEventRecord(e0, 0) == cudaSuccess;
        for (int i = 0; i < reps && ok; ++i)
            ok = run_unchecked(p, a, b, 0, -1) == MOA_OK;
        ok = ok && cudaEventRecord(e1, 0) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
        float t = 0.f;
        if (ok && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess)
            ms = t / reps;
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    cudaFree(a);
    cudaFree(b);
    return ms;
}

bool autotune_enabled() { return env_int("MOA_AUTOTUNE", 1) != 0; }
bool env_set(const char *name)
{
    const char *v = std::getenv(name);
    return v && *v;
}

moa_status_t run(moa_fft_plan_s *p, const void *in, void *out, void *stream, int sign)
{
    if (!is_live(p))
        return MOA_ERR_INVALID_ARG;
    moa_status_t st = check_io(in, out);
    if (st != MOA_OK)
        return st;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t np = p->batched ? 1 : p->passes.size();
    for (size_t i = 0; i < np; ++i)
        if ((st = run_pass(p, i, in, out, s, sign)) != MOA_OK)
            return st;
    return MOA_OK;
}


// Build a plan (not yet registered) with optional fixed choices.
// Kernel that runs pass d of plan p (the name moa_fft_pass_info reports).
void pass_name(const moa_fft_plan_s *p, const PassDesc &d, char *buf, size_t len)
{
    if (p->batched)
        snprintf(buf, len, "batched_kernel");
    else if (d.kind == moa::PASS_TC)
        snprintf(buf, len, d.umma ? "tc_umma_kernel<%d,%d>" : "tc_row_kernel<%d,%d>",
                 p->dtype == MOA_C64_TC_BF16 ? 1 : 0, d.logN);
    else if (d.kind == moa::PASS_LIFT3)
        snprintf(buf, len, "lift3_kernel<%d,%d>", d.logF, d.logN);
    else if (d.kind == moa::PASS_PLANE1)
        snprintf(buf, len, "plane3d_p1_kernel");
    // N = 4096 column passes run two columns per thread (four with MOA_COL2=0,
    // or on an output that is only 8-byte aligned)
    else if (d.kind == moa::PASS_PLANE2)
        snprintf(buf, len, moa::pipe_col2_active() ? "pipe_col2_kernel<0,3>" : "pipe_col_kernel<12,0,3>");
    else if (d.pipe && (d.kind == moa::PASS_COL || d.blk == 2) && d.logN == 12 && moa::pipe_col2_active())
        snprintf(buf, len, "pipe_col2_kernel<%d,%d>", d.tw4, d.blk);
    else if (d.pipe && (d.kind == moa::PASS_COL || d.blk == 2))
        snprintf(buf, len, "pipe_col_kernel<%d,%d,%d>", d.logN, d.tw4, d.blk);
    else if (d.pipe)
        snprintf(buf, len, "pipe_rowT_kernel<%d>", d.logN);
    else if (d.sched == 3)
        snprintf(buf, len, "row_warp_kernel<%d>", d.logN);
    else if (d.kind == moa::PASS_COL && d.sched > 0)
        snprintf(buf, len, "col_pass_kernel<%d,%d,%d>", d.logN, d.tw4, d.sched);
    else if (d.kind == moa::PASS_COL)
        snprintf(buf, len, "col_pass_kernel<%d,%d>", d.logN, d.tw4);
    else if (d.sched > 0)
        snprintf(buf, len, "row_pass_kernel<%d,%d,%d>", d.logN, d.Rt > 1 ? 1 : 0, d.sched);
    else
        snprintf(buf, len, "row_pass_kernel<%d,%d>", d.logN, d.Rt > 1 ? 1 : 0);
}

// MOA_LOG=1: plan decisions and autotuner timings on stderr.
bool log_enabled() { return env_int("MOA_LOG", 0) == 1; }

void log_plan(const moa_fft_plan_s *p, const char *how)
{
    if (!log_enabled())
        return;
    std::string dims;
    if (p->batched) {
        dims = "batched: " + std::to_string(p->bl.ntasks) + " tasks";
    } else {
        for (int i = 0; i < p->dims; ++i)
            dims += (i ? "x" : "") + std::to_string(p->n[i]);
        dims += " batch " + std::to_string(p->batch);
    }
    std::string passes;
    const size_t np = p->batched ? 1 : p->passes.size();
    for (size_t i = 0; i < np; ++i) {
        char buf[64];
        pass_name(p, p->batched ? PassDesc{} : p->passes[i], buf, sizeof(buf));
        passes += (i ? " -> " : "") + std::string(buf);
    }
    fprintf(stderr, "moafft: plan %s sign %+d dtype %d (%s): split r=%lld c=%lld, workspace %zu bytes, %s\n",
            dims.c_str(), p->sign, p->dtype, how, (long long)p->split_r, (long long)p->split_c, p->workspace_bytes,
            passes.c_str());
}

// Choices a plan may have fixed (the autotuner's candidates); -1 = default
// or environment override.
struct PlanOpts {
    int lr = -1, pipe = -1, lift3 = -1, tile = -1, two_pass3d = -1, sched = -1;
};

moa_status_t make_plan(moa_fft_plan_s **out, const int64_t *n, int dims, int64_t batch, int sign, int dtype,
                       int64_t total, const PlanOpts &o)
{
    *out = nullptr;
    moa_fft_plan_s *p = new (std::nothrow) moa_fft_plan_s();
    if (!p)
        return MOA_ERR_ALLOC;
    p->dims = dims;
    for (int i = 0; i < dims; ++i)
        p->n[i] = n[i];
    p->batch = batch;
    p->sign = sign;
    p->dtype = dtype;
    p->total = total;
    p->opt_lr = o.lr;
    p->opt_pipe = o.pipe;
    p->opt_lift3 = o.lift3;
    p->opt_tile = o.tile;
    p->opt_3d2 = o.two_pass3d;
    p->opt_sched = o.sched;
    p->tma = moa::pipe_supported();
    p->fault_wait = env_int("MOA_FAULT_WAIT", 0) == 1;
    moa_status_t st = build_passes(p);
    if (st == MOA_OK) {
        assign_pipe(p);
        assign_sched(p);
        st = allocate_and_fill(p);
    }
    if (st != MOA_OK) {
        free_plan_memory(p);
        delete p;
        return st;
    }
    *out = p;
    return MOA_OK;
}

moa_status_t make_batched(moa_fft_plan_s **out, const int64_t *lengths, int64_t count, int sign, int dtype,
                          const int *dlr)
{
    *out = nullptr;
    moa_fft_plan_s *p = new (std::nothrow) moa_fft_plan_s();
    if (!p)
        return MOA_ERR_ALLOC;
    p->sign = sign;
    p->dtype = dtype;
    for (int l = 0; l <= 16; ++l)
        p->opt_batch_dlr[l] = dlr[l];
    const moa_status_t st = build_batched(p, lengths, count);
    if (st != MOA_OK) {
        free_plan_memory(p);
        delete p;
        return st;
    }
    *out = p;
    return MOA_OK;
}

// What distinguishes two plans for timing: every pass's kernel and tile.
std::string plan_signature(const moa_fft_plan_s *p)
{
    std::string sig;
    for (const PassDesc &d : p->passes) {
        char buf[96];
        pass_name(p, d, buf, sizeof(buf));
        sig += std::string(buf) + "/" + std::to_string(d.logF) + ";";
    }
    return sig;
}

// Short description of a plan's choices (log lines and moa_fft_plan_choice).
std::string plan_choice(const moa_fft_plan_s *p)
{
    std::string c;
    if (p->batched) {
        c = "batched: log2 r offset per length";
        for (int l = 13; l <= 16; ++l)
            c += " 2^" + std::to_string(l) + ":" + std::to_string(p->opt_batch_dlr[l]);
    } else {
        c = "split r=" + std::to_string((long long)p->split_r) + " c=" + std::to_string((long long)p->split_c) +
            ", tile 2^" + std::to_string(tile_or_default(p->opt_tile)) + ", passes ";
        for (size_t i = 0; i < p->passes.size(); ++i) {
            char buf[96];
            pass_name(p, p->passes[i], buf, sizeof(buf));
            c += (i ? " -> " : "") + std::string(buf);
        }
    }
    return c + " (" + p->how + ")";
}

}  // namespace

// Argument checks shared by moa_fft_plan and moa_fft_estimate; *total gets
// the complex elements per exec.
moa_status_t validate_request(const int64_t *n, int dims, int64_t batch, int sign, int dtype, int64_t *total)
{
    if (!n || dims < 1 || dims > 3 || batch < 1 || (sign != 1 && sign != -1))
        return MOA_ERR_INVALID_ARG;
    if (dtype != MOA_C64 && dtype != MOA_C64_TC_FP16 && dtype != MOA_C64_TC_BF16)
        return MOA_ERR_INVALID_ARG;
    int64_t t = batch;
    for (int i = 0; i < dims; ++i) {
        if (!pow2_ge2(n[i]))
            return MOA_ERR_INVALID_SIZE;
        if (n[i] > (int64_t(1) << (dims == 1 ? 30 : 24)))
            return MOA_ERR_UNSUPPORTED;
        t *= n[i];
        if (t >= (int64_t(1) << 31))
            return MOA_ERR_UNSUPPORTED;
    }
    // the tensor-core path covers 1-D transforms of 256 or 4096 points
    if (dtype != MOA_C64 && !(dims == 1 && (n[0] == 256 || n[0] == 4096)))
        return MOA_ERR_UNSUPPORTED;
    *total = t;
    return MOA_OK;
}

extern "C" {

moa_status_t moa_fft_plan(moa_fft_plan_t *plan, const int64_t *n, int dims, int64_t batch, int sign, int dtype)
{
    if (!plan)
        return MOA_ERR_INVALID_ARG;
    *plan = nullptr;
    int64_t total = 0;
    if (const moa_status_t vs = validate_request(n, dims, batch, sign, dtype, &total))
        return vs;

    // The autotuner (Sec. 4.8: every breakpoint is correct; the choice is
    // made by timing, as the paper's script-based search does): every
    // admissible r x c split of a lifted 1-D transform and its three-level
    // lift, the pipelined or generic strided kernels, the tile size of the
    // generic passes, and for 256^3 arrays the two-pass or per-axis form;
    // then, on the best of those, the radix schedule of the generic passes
    // (small radix first or last, radix-8 stages, warp-shuffle rows).
    // Candidates that build the same passes are timed once.  A choice fixed
    // by an environment override is not searched.
    PlanOpts best_opts;
    const int L = ilog2(n[0]);
    std::string how = "defaults or environment overrides";
    const bool lifted = dims == 1 && L > 12;
    const bool tunable = dtype == MOA_C64 && autotune_enabled() && (dims > 1 || lifted || batch > 1);
    if (tunable) {
        // the key names the choices fixed by environment overrides, which
        // are not searched (their cached entry holds -1 = default there)
        std::string key = device_tag() + ":plan:" + std::to_string(dims);
        for (int i = 0; i < dims; ++i)
            key += ":" + std::to_string((long long)n[i]);
        key += ":" + std::to_string((long long)batch) + ":";
        const char *fixed[] = {"MOA_SPLIT_LOG2R", "MOA_LIFT3", "MOA_PIPE", "MOA_TILE_LOG2", "MOA_3D_TWO_PASS",
                               "MOA_SCHED"};
        for (int i = 0; i < 6; ++i)
            key += env_set(fixed[i]) ? "f" : "s";
        std::string v;
        PlanOpts c;
        if (tune_get(key, v) && sscanf(v.c_str(), "%d %d %d %d %d %d", &c.lr, &c.pipe, &c.lift3, &c.tile,
                                       &c.two_pass3d, &c.sched) == 6) {
            best_opts = c;
            how = "autotuner choice from the cache";
        } else {
            how = "autotuned";
            std::vector<int> lrs{-1}, pipes{-1}, lift3s{-1}, tiles{-1}, twos{-1};
            if (lifted && L <= 24 && !env_set("MOA_SPLIT_LOG2R") && !env_set("MOA_LIFT3")) {
                lrs.clear();
                for (int lr = std::max(1, L - 12); lr <= std::min(12, L - 1); ++lr)
                    lrs.push_back(lr);
                lift3s = {0};
            }
            if (!env_set("MOA_PIPE"))
                pipes = {2, 1, 0};
            if (!env_set("MOA_TILE_LOG2"))
                tiles = {12, 11, 13};
            if (dims == 3 && !env_set("MOA_3D_TWO_PASS"))
                twos = {1, 0};
            std::vector<PlanOpts> cands;
            for (int lr : lrs)
                for (int pipe : pipes)
                    for (int tile : tiles)
                        for (int two : twos) {
                            PlanOpts o;
                            o.lr = lr;
                            o.pipe = pipe;
                            o.lift3 = lift3s[0];
                            o.tile = tile;
                            o.two_pass3d = two;
                            cands.push_back(o);
                        }
            if (lifted && L >= 21 && L <= 24 && !env_set("MOA_SPLIT_LOG2R") && !env_set("MOA_LIFT3"))
                for (int tile : tiles) {
                    PlanOpts o;
                    o.lift3 = 1;
                    o.tile = tile;
                    cands.push_back(o);
                }
            float best = INFINITY;
            std::set<std::string> seen;
            // time one candidate (once per distinct pass list); false on a hard error
            moa_status_t err = MOA_OK;
            auto consider = [&](const PlanOpts &o) {
                moa_fft_plan_s *cand = nullptr;
                const moa_status_t st = make_plan(&cand, n, dims, batch, sign, dtype, total, o);
                if (st == MOA_ERR_UNSUPPORTED)
                    return true;
                if (st != MOA_OK) {
                    err = st;
                    return false;
                }
                const std::string sig = plan_signature(cand);
                if (!seen.insert(sig).second) {   // the same passes as a candidate already timed
                    free_plan_memory(cand);
                    delete cand;
                    return true;
                }
                const float ms = time_exec(cand);
                if (log_enabled())
                    fprintf(stderr, "moafft: autotune candidate %s: %.1f us\n", sig.c_str(), ms * 1e3f);
                free_plan_memory(cand);
                delete cand;
                if (ms < best) {
                    best = ms;
                    best_opts = o;
                }
                return true;
            };
            for (const PlanOpts &o : cands)
                if (!consider(o))
                    return err;
            // then the radix schedule of the generic passes, on the best plan
            // (schedules that change no pass give the same pass list and are
            // not timed again)
            if (!env_set("MOA_SCHED") && std::isfinite(best)) {
                const PlanOpts base = best_opts;
                for (int sc = 1; sc <= 3; ++sc) {
                    PlanOpts o = base;
                    o.sched = sc;
                    if (!consider(o))
                        return err;
                }
            }
            if (std::isfinite(best))
                tune_put(key, std::to_string(best_opts.lr) + " " + std::to_string(best_opts.pipe) + " " +
                                  std::to_string(best_opts.lift3) + " " + std::to_string(best_opts.tile) + " " +
                                  std::to_string(best_opts.two_pass3d) + " " + std::to_string(best_opts.sched));
        }
    }
    moa_fft_plan_s *p = nullptr;
    const moa_status_t st = make_plan(&p, n, dims, batch, sign, dtype, total, best_opts);
    if (st != MOA_OK)
        return st;
    p->how = how;
    log_plan(p, how.c_str());
    {
        std::lock_guard<std::mutex> lk(g_plans_mu);
        g_plans.insert(p);
    }
    *plan = p;
    return MOA_OK;
}

moa_status_t moa_fft_plan_batched(moa_fft_plan_t *plan, const int64_t *lengths, int64_t count, int sign,
                                  int dtype)
{
    if (!plan)
        return MOA_ERR_INVALID_ARG;
    *plan = nullptr;
    if (!lengths || count < 1 || (sign != 1 && sign != -1))
        return MOA_ERR_INVALID_ARG;
    if (dtype != MOA_C64 && dtype != MOA_C64_TC_FP16 && dtype != MOA_C64_TC_BF16)
        return MOA_ERR_INVALID_ARG;
    int64_t total = 0;
    for (int64_t i = 0; i < count; ++i) {
        if (!pow2_ge2(lengths[i]))
            return MOA_ERR_INVALID_SIZE;
        if (lengths[i] > 65536)
            return MOA_ERR_UNSUPPORTED;
        total += lengths[i];
        if (total >= (int64_t(1) << 31))
            return MOA_ERR_UNSUPPORTED;
    }
    if (dtype != MOA_C64)
        return MOA_ERR_UNSUPPORTED;
    // per-length split of the large transforms (log2 r offset -1, 0 or +1
    // from floor(log2 n / 2)), one length at a time, the others held at their
    // best so far
    int dlr[17] = {0};
    int hist[17] = {0};
    for (int64_t i = 0; i < count; ++i)
        hist[ilog2(lengths[i])]++;
    const bool any_large = hist[13] + hist[14] + hist[15] + hist[16] > 0;
    std::string how = "default split of the large transforms";
    if (any_large && autotune_enabled() && !env_set("MOA_BATCH_LOG2R")) {
        std::string key = device_tag() + ":batched2:";
        for (int l = 1; l <= 16; ++l)
            key += std::to_string(hist[l]) + (l < 16 ? "," : "");
        std::string v;
        int c[4];
        if (tune_get(key, v) && sscanf(v.c_str(), "%d %d %d %d", &c[0], &c[1], &c[2], &c[3]) == 4) {
            for (int l = 13; l <= 16; ++l)
                dlr[l] = c[l - 13];
            how = "autotuner choice from the cache";
        } else {
            how = "autotuned";
            auto timed = [&](const int *off, float &ms) -> moa_status_t {
                moa_fft_plan_s *cand = nullptr;
                const moa_status_t st = make_batched(&cand, lengths, count, sign, dtype, off);
                if (st != MOA_OK)
                    return st;
                ms = time_exec(cand);
                if (log_enabled())
                    fprintf(stderr,
                            "moafft: autotune batched (%lld transforms): log2 r offsets 2^13:%+d 2^14:%+d 2^15:%+d "
                            "2^16:%+d: %.1f us\n",
                            (long long)count, off[13], off[14], off[15], off[16], ms * 1e3f);
                free_plan_memory(cand);
                delete cand;
                return MOA_OK;
            };
            float best = INFINITY;
            moa_status_t st = timed(dlr, best);
            if (st != MOA_OK)
                return st;
            for (int l = 13; l <= 16; ++l) {
                if (hist[l] == 0)
                    continue;
                for (int d = -1; d <= 1; d += 2) {
                    int off[17];
                    std::copy(dlr, dlr + 17, off);
                    off[l] = d;
                    float ms = INFINITY;
                    if ((st = timed(off, ms)) != MOA_OK)
                        return st;
                    if (ms < best) {
                        best = ms;
                        dlr[l] = d;
                    }
                }
            }
            if (std::isfinite(best))
                tune_put(key, std::to_string(dlr[13]) + " " + std::to_string(dlr[14]) + " " +
                                  std::to_string(dlr[15]) + " " + std::to_string(dlr[16]));
        }
    }
    moa_fft_plan_s *p = nullptr;
    const moa_status_t st = make_batched(&p, lengths, count, sign, dtype, dlr);
    if (st != MOA_OK)
        return st;
    p->how = how;
    log_plan(p, how.c_str());
    {
        std::lock_guard<std::mutex> lk(g_plans_mu);
        g_plans.insert(p);
    }
    *plan = p;
    return MOA_OK;
}

moa_status_t moa_fft_exec(moa_fft_plan_t plan, const void *in, void *out, void *stream)
{
    if (!is_live(plan))
        return MOA_ERR_INVALID_ARG;
    return run(plan, in, out, stream, plan->sign);
}

moa_status_t moa_fft_exec_adjoint(moa_fft_plan_t plan, const void *in, void *out, void *stream)
{
    if (!is_live(plan))
        return MOA_ERR_INVALID_ARG;
    return run(plan, in, out, stream, -plan->sign);
}

moa_status_t moa_fft_exec_pass(moa_fft_plan_t plan, int index, int sign, const void *in, void *out,
                               void *stream)
{
    if (!is_live(plan) || (sign != 1 && sign != -1))
        return MOA_ERR_INVALID_ARG;
    if (index < 0 || (size_t)index >= (plan->batched ? 1 : plan->passes.size()))
        return MOA_ERR_INVALID_ARG;
    moa_status_t st = check_io(in, out);
    if (st != MOA_OK)
        return st;
    return run_pass(plan, (size_t)index, in, out, static_cast<cudaStream_t>(stream), sign);
}

moa_status_t moa_fft_exec_host(moa_fft_plan_t plan, const void *host_in, void *host_out, void *dev_buf,
                               void *stream)
{
    if (!is_live(plan))
        return MOA_ERR_INVALID_ARG;
    if (!host_in || !host_out || !dev_buf)
        return MOA_ERR_INVALID_ARG;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)plan->total * sizeof(float2);
    if (cudaMemcpyAsync(dev_buf, host_in, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return MOA_ERR_CUDA;
    moa_status_t st = run(plan, dev_buf, dev_buf, stream, plan->sign);
    if (st != MOA_OK)
        return st;
    if (cudaMemcpyAsync(host_out, dev_buf, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return MOA_ERR_CUDA;
    return MOA_OK;
}

moa_status_t moa_fft_status(moa_fft_plan_t plan)
{
    if (!is_live(plan))
        return MOA_ERR_INVALID_ARG;
    int h = 0;
    if (cudaMemcpy(&h, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return MOA_ERR_CUDA;
    if (h != 0 && cudaMemset(plan->d_status, 0, sizeof(int)) != cudaSuccess)
        return MOA_ERR_CUDA;
    return static_cast<moa_status_t>(h);
}

const char *moa_fft_error_string(moa_status_t status)
{
    switch (status) {
    case MOA_OK: return "success";
    case MOA_ERR_INVALID_ARG: return "invalid argument";
    case MOA_ERR_INVALID_SIZE: return "invalid size (lengths must be powers of two >= 2)";
    case MOA_ERR_UNSUPPORTED: return "unsupported configuration";
    case MOA_ERR_ALLOC: return "allocation failed";
    case MOA_ERR_CUDA: return "CUDA runtime error";
    case MOA_ERR_TIMEOUT: return "device-side wait timed out";
    default: return "unknown status";
    }
}

moa_status_t moa_fft_plan_info(moa_fft_plan_t plan, int *passes, int64_t *split_r, int64_t *split_c,
                               size_t *workspace_bytes)
{
    if (!is_live(plan))
        return MOA_ERR_INVALID_ARG;
    if (passes)
        *passes = plan->batched ? 1 : (int)plan->passes.size();
    if (split_r)
        *split_r = plan->split_r;
    if (split_c)
        *split_c = plan->split_c;
    if (workspace_bytes)
        *workspace_bytes = plan->workspace_bytes;
    return MOA_OK;
}

moa_status_t moa_fft_plan_choice(moa_fft_plan_t plan, char *text, size_t text_len)
{
    if (!is_live(plan) || !text || text_len == 0)
        return MOA_ERR_INVALID_ARG;
    const std::string c = plan_choice(plan);
    snprintf(text, text_len, "%s", c.c_str());
    return MOA_OK;
}

moa_status_t moa_fft_pass_info(moa_fft_plan_t plan, int index, char *name, size_t name_len, int64_t *bytes)
{
    if (!is_live(plan) || index < 0 || (size_t)index >= (plan->batched ? 1 : plan->passes.size()))
        return MOA_ERR_INVALID_ARG;
    if (name_len > 0 && !name)
        return MOA_ERR_INVALID_ARG;
    char buf[64];
    const PassDesc d = plan->batched ? PassDesc{} : plan->passes[index];
    pass_name(plan, d, buf, sizeof(buf));
    if (name_len > 0) {
        strncpy(name, buf, name_len - 1);
        name[name_len - 1] = '\0';
    }
    if (bytes)
        *bytes = 2 * (int64_t)sizeof(float2) * plan->total;
    return MOA_OK;
}

moa_status_t moa_fft_batched_queue(const int64_t *lengths, int64_t count, int64_t resident, int64_t *order,
                                   int32_t *tasks, int64_t capacity, int64_t *ntasks)
{
    if (!lengths || count < 1 || resident < 1 || capacity < 0 || (capacity > 0 && !tasks))
        return MOA_ERR_INVALID_ARG;
    int64_t total = 0;
    for (int64_t i = 0; i < count; ++i) {
        if (!pow2_ge2(lengths[i]))
            return MOA_ERR_INVALID_SIZE;
        if (lengths[i] > 65536)
            return MOA_ERR_UNSUPPORTED;
        total += lengths[i];
        if (total >= (int64_t(1) << 31))
            return MOA_ERR_UNSUPPORTED;
    }
    BatchQueue bq;
    const int no_offsets[17] = {0};
    build_queue(lengths, count, no_offsets, resident, bq);
    const int64_t nt = (int64_t)bq.queue.size();
    if (ntasks)
        *ntasks = nt;
    if (order) {
        // offsets grow with the input index, so each sorted offset maps back by search
        std::vector<int64_t> offset(count);
        int64_t o = 0;
        for (int64_t i = 0; i < count; ++i) {
            offset[i] = o;
            o += lengths[i];
        }
        for (int64_t k = 0; k < count; ++k)
            order[k] = std::lower_bound(offset.begin(), offset.end(), bq.offs_sorted[k]) - offset.begin();
    }
    if (capacity == 0)
        return MOA_OK;
    if (capacity < nt)
        return MOA_ERR_INVALID_ARG;
    for (int64_t t = 0; t < nt; ++t) {
        const moa::BatchTask &q = bq.queue[t];
        int32_t *d = tasks + 6 * t;
        d[0] = q.first;
        d[1] = q.count;
        d[2] = q.tile;
        d[3] = q.logn;
        d[4] = q.logr;
        d[5] = q.kind;
    }
    return MOA_OK;
}

moa_status_t moa_fft_plan_table(moa_fft_plan_t plan, int table, int index, void *host_out, int64_t capacity,
                                int64_t *entries)
{
    if (!is_live(plan) || plan->batched)
        return MOA_ERR_INVALID_ARG;
    const float2 *src = nullptr;
    int64_t count = 0;
    if (table == 0) {
        if (index < 1 || index > 12 || !plan->tw.stage[index])
            return MOA_ERR_INVALID_ARG;
        src = plan->tw.stage[index];
        count = moa::stage_table_entries(index);
    } else if (table >= 3 && table <= 5) {
        const int v = table - 2;
        if (index < 1 || index > 12 || !plan->tw.vstage[v][index])
            return MOA_ERR_INVALID_ARG;
        src = plan->tw.vstage[v][index];
        count = moa::stage_table_entries(index, v);
    } else if (table == 1 || table == 2) {
        if (!plan->tw.lo || !plan->tw.hi)
            return MOA_ERR_INVALID_ARG;
        const int logn = ilog2(plan->total / plan->batch);
        src = table == 1 ? plan->tw.lo : plan->tw.hi;
        count = table == 1 ? (int64_t(1) << plan->tw.h) : (int64_t(1) << (logn - plan->tw.h));
    } else {
        return MOA_ERR_INVALID_ARG;
    }
    if (entries)
        *entries = count;
    if (!host_out)
        return capacity == 0 ? MOA_OK : MOA_ERR_INVALID_ARG;
    if (capacity < count)
        return MOA_ERR_INVALID_ARG;
    if (count > 0 && cudaMemcpy(host_out, src, (size_t)count * sizeof(float2), cudaMemcpyDeviceToHost) != cudaSuccess)
        return MOA_ERR_CUDA;
    return MOA_OK;
}

moa_status_t moa_fft_estimate(const int64_t *n, int dims, int64_t batch, int dtype, int tma, int *passes,
                              int64_t *split_r, int64_t *split_c, size_t *workspace_bytes, char *kernels,
                              size_t kernels_len)
{
    if (tma < -1 || tma > 1 || (kernels_len > 0 && !kernels))
        return MOA_ERR_INVALID_ARG;
    int64_t total = 0;
    if (const moa_status_t vs = validate_request(n, dims, batch, -1, dtype, &total))
        return vs;
    moa_fft_plan_s p;   // host description only: nothing is allocated or launched
    p.dims = dims;
    for (int i = 0; i < dims; ++i)
        p.n[i] = n[i];
    p.batch = batch;
    p.dtype = dtype;
    p.total = total;
    p.tma = tma < 0 ? moa::pipe_supported() : tma == 1;
    if (const moa_status_t st = build_passes(&p))
        return st;
    assign_pipe(&p);
    assign_sched(&p);
    if (passes)
        *passes = (int)p.passes.size();
    if (split_r)
        *split_r = p.split_r;
    if (split_c)
        *split_c = p.split_c;
    if (workspace_bytes)
        *workspace_bytes = p.workspace_bytes;
    if (kernels_len > 0) {
        std::string all;
        for (size_t i = 0; i < p.passes.size(); ++i) {
            char buf[64];
            pass_name(&p, p.passes[i], buf, sizeof(buf));
            all += (i ? ";" : "") + std::string(buf);
        }
        strncpy(kernels, all.c_str(), kernels_len - 1);
        kernels[kernels_len - 1] = '\0';
    }
    return MOA_OK;
}

moa_status_t moa_fft_destroy(moa_fft_plan_t plan)
{
    if (!plan)
        return MOA_OK;
    {
        std::lock_guard<std::mutex> lk(g_plans_mu);
        if (!g_plans.erase(plan))
            return MOA_ERR_INVALID_ARG;
    }
    free_plan_memory(plan);
    delete plan;
    return MOA_OK;
}

}  // extern "C"
