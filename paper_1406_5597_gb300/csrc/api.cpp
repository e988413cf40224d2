// Host side of libfft3d: plan construction (size checks, pass selection,
// FP64 twiddle tables), the C ABI declared in include/fft3d.h, and the pass
// sequences of the forward and inverse transforms.
//
// Forward (Sec. 2.1 steps 1 and 3, with the n0 step done in place at its
// natural stride as Sec. 2.2 proposes):
//   1. n2 rows:   real rows -> half-spectrum rows          (in  -> out)
//   2. n1 axis:   c2c at stride H per (j0, k2)             (out, in place)
//   3. n0 axis:   c2c at stride n1*H per flat (k1, k2)     (out, in place)
// Inverse: the same steps in reverse order (Sec. 2.1), on the clobbered input.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include <cuda_bf16.h>
#include <nvtx3/nvToolsExt.h>
#include <cuda_fp16.h>

#include "args.h"
#include "energy.h"
#include "fft3d.h"
#include "cplane.h"
#include "group_wt.h"
#include "ns.h"
#include "plane.h"
#include "tma_host.h"

namespace fft3d {
const LenEntry* entries_small(int* n);
const LenEntry* entries_mixed(int* n);
const LenEntry* entries_256_512(int* n);
const LenEntry* entries_1024_2048(int* n);
const LenEntry* entries_mixed_wide(int* n);
cudaError_t launch_swap01(const float2* in, float2* out, long long batch, long long n0, long long n1, long long H,
                          cudaStream_t s);

const LenEntry* find_len(int L)
{
    using Fn = const LenEntry* (*)(int*);
    static const Fn groups[] = {entries_small, entries_mixed, entries_256_512, entries_1024_2048, entries_mixed_wide};
    for (Fn f : groups) {
        int n = 0;
        const LenEntry* e = f(&n);
        for (int i = 0; i < n; ++i)
            if (e[i].L == L) return &e[i];
    }
    return nullptr;
}
}  // namespace fft3d

using namespace fft3d;

namespace {

constexpr int kMaxAxis = 4096;
thread_local int g_last_error = FFT3D_OK;

int fail(int status)
{
    g_last_error = status;
    return status;
}

// FFT3D_LOG=1: planner and autotuner decisions on stderr.
bool log_enabled()
{
    static const bool on = [] {
        const char* v = std::getenv("FFT3D_LOG");
        return v && *v && std::strcmp(v, "0") != 0;
    }();
    return on;
}

// FFT3D_FORCE_PASSES: a test / benchmark override of the planner, read at every
// plan creation: comma-separated forms OR-ed into the flags of every FP32 plan
// ("three", "generic", "fused", "cluster", "transpose", "transpose_back";
// unknown names are ignored).  Combinations that are invalid for a plan fail
// as if passed as flags.
int forced_flags()
{
    const char* v = std::getenv("FFT3D_FORCE_PASSES");
    if (!v) return 0;
    static const struct {
        const char* name;
        int flags;
    } forms[] = {{"three", FFT3D_FLAG_THREE_PASS},
                 {"generic", FFT3D_FLAG_GENERIC},
                 {"fused", FFT3D_FLAG_FUSED_PLANE},
                 {"cluster", FFT3D_FLAG_CLUSTER_PLANE},
                 {"transpose", FFT3D_FLAG_EXPLICIT_TRANSPOSE},
                 {"transpose_back", FFT3D_FLAG_EXPLICIT_TRANSPOSE | FFT3D_FLAG_TRANSPOSE_BACK}};
    int f = 0;
    std::string s(v);
    size_t pos = 0;
    while (pos <= s.size()) {
        const size_t end = s.find(',', pos) == std::string::npos ? s.size() : s.find(',', pos);
        const std::string tok = s.substr(pos, end - pos);
        for (const auto& m : forms)
            if (tok == m.name) f |= m.flags;
        pos = end + 1;
    }
    return f;
}

bool smooth2357(long long n)
{
    if (n < 1) return false;
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}

// exp(+2 pi i m / L) in FP64 with exact quarter-turn reduction:
// 2 pi m / L = (pi/2) (q + r/L), q = floor(4m/L); the residual angle is taken
// from the nearer end of [0, pi/2] so that the argument passed to cos/sin is
// at most pi/4.  Quarter-turn points come out exactly (0, +-1).
void root_of_unity(long long m, long long L, double* c, double* s)
{
    m %= L;
    if (m < 0) m += L;
    const long long q = (4 * m) / L;
    const long long r = 4 * m - q * L;  // in [0, L)
    const double half_pi = 1.57079632679489661923;
    double c0, s0;
    if (2 * r <= L) {
        const double a = half_pi * (double)r / (double)L;
        c0 = std::cos(a);
        s0 = std::sin(a);
    } else {
        const double a = half_pi * (double)(L - r) / (double)L;
        c0 = std::sin(a);
        s0 = std::cos(a);
    }
    switch (q & 3) {
    case 0: *c = c0; *s = s0; break;
    case 1: *c = -s0; *s = c0; break;
    case 2: *c = -c0; *s = -s0; break;
    default: *c = s0; *s = -c0; break;
    }
}

// Forward-sign table W_L^m = exp(-2 pi i m / L), m in [0, count), rounded to FP32.
std::vector<float2> forward_table(long long L, long long count)
{
    std::vector<float2> t((size_t)count);
    for (long long m = 0; m < count; ++m) {
        double c, s;
        root_of_unity(m, L, &c, &s);
        t[(size_t)m] = make_float2((float)c, (float)(-s));
    }
    return t;
}

// Stockham radices of a 2357-smooth length; no stages (nst = 0) for any other
// length, which runs in Bluestein form (setup_bluestein).
GenPlan generic_radices(int L)
{
    GenPlan g{};
    g.L = L;
    if (!smooth2357(L)) return g;
    int rem = L;
    while (rem > 1) {
        int R = 0;
        for (int cand : {8, 4, 2, 3, 5, 7})
            if (rem % cand == 0) { R = cand; break; }
        g.radix[g.nst++] = R;
        rem /= R;
    }
    return g;
}

struct Axis {
    int L = 1;
    const LenEntry* spec = nullptr;
    const TcEntry* tc = nullptr;  // tensor-core radix-16 column kernel (TC dtypes)
    const SplitEntry* split[2] = {nullptr, nullptr};  // cluster-split column kernels of this length
    const TmaSplitEntry* tsplit = nullptr;             // TMA-fed cluster split of this length
    const L2SplitEntry* l2split = nullptr;             // residue split through L2 of this length
    float2* d_l2scratch = nullptr;                     // its scratch (the plan's, shared by both axes)
    int l2_ctas = 0;
    GenPlan gen{};
    float2* d_tw = nullptr;
    float2* d_blu = nullptr;  // Bluestein tables (chirp, bhat, W_M), lengths with a prime factor above 7
    // FFT3D_F64 plans: the same tables in FP64
    GenPlan64 gen64{};
    double2* d_tw64 = nullptr;
    double2* d_blu64 = nullptr;
};

bool is_tc_dtype(int dtype) { return dtype == FFT3D_F32_TC_BF16X3 || dtype == FFT3D_F32_TC_F16; }

cudaError_t upload(const std::vector<float2>& h, float2** d);

int next_pow2(int n)
{
    int m = 1;
    while (m < n) m <<= 1;
    return m;
}

// In-place forward (negative-sign) FFT of a power-of-two length in FP64:
// bit-reversal permutation, then radix-2 butterflies of growing span.
void fft_pow2_fp64(std::vector<double>& re, std::vector<double>& im)
{
    const int n = (int)re.size();
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            std::swap(re[i], re[j]);
            std::swap(im[i], im[j]);
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        const int half = len / 2;
        for (int k = 0; k < half; ++k) {
            double c, s;
            root_of_unity(k, len, &c, &s);
            const double wr = c, wi = -s;  // W_len^k = exp(-2 pi i k / len)
            for (int i = k; i < n; i += len) {
                const int j = i + half;
                const double tr = re[j] * wr - im[j] * wi, ti = re[j] * wi + im[j] * wr;
                re[j] = re[i] - tr;
                im[j] = im[i] - ti;
                re[i] += tr;
                im[i] += ti;
            }
        }
    }
}

// Forward-sign table W_L^m, m in [0, count), in FP64.
std::vector<double2> forward_table64(long long L, long long count)
{
    std::vector<double2> t((size_t)count);
    for (long long m = 0; m < count; ++m) {
        double c, s;
        root_of_unity(m, L, &c, &s);
        t[(size_t)m] = make_double2(c, -s);
    }
    return t;
}

cudaError_t upload64(const std::vector<double2>& h, double2** d)
{
    cudaError_t e = cudaMalloc((void**)d, h.size() * sizeof(double2));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*d, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice);
}

// The FP64 chirp, transformed chirp and length-M table of a Bluestein axis
// (exactly as setup_bluestein, without the rounding to FP32).
struct BluesteinTables {
    int M;
    std::vector<double2> chirp, bhat, tw;
};
BluesteinTables bluestein_tables(int L);

// Bluestein form of a length-L axis (L has a prime factor above 7): M is the
// smallest power of two >= 2L - 1, and one device array holds, rounded to FP32
// from FP64, the chirp c[n] = exp(-i pi n^2 / L) (n^2 reduced mod 2L, so the
// angle is exact), bhat = (1/M) FFT_M(b) with b[m] = b[M - m] = conj(c[m]) for
// m < L (zero elsewhere), and the length-M forward table.
BluesteinTables bluestein_tables(int L)
{
    BluesteinTables t;
    const int M = next_pow2(2 * L - 1);
    t.M = M;
    t.chirp.resize((size_t)L);
    t.bhat.resize((size_t)M);
    std::vector<double> br((size_t)M, 0.0), bi((size_t)M, 0.0);
    for (long long n = 0; n < L; ++n) {
        double c, s;
        root_of_unity((n * n) % (2LL * L), 2LL * L, &c, &s);  // exp(+i pi n^2 / L) = conj(c[n])
        t.chirp[(size_t)n] = make_double2(c, -s);
        br[(size_t)n] = c;
        bi[(size_t)n] = s;
        if (n > 0) {
            br[(size_t)(M - n)] = c;
            bi[(size_t)(M - n)] = s;
        }
    }
    fft_pow2_fp64(br, bi);
    for (int k = 0; k < M; ++k) t.bhat[(size_t)k] = make_double2(br[k] / M, bi[k] / M);
    t.tw = forward_table64(M, M);
    return t;
}

cudaError_t setup_bluestein(Axis& a)
{
    const int L = a.L;
    const BluesteinTables t = bluestein_tables(L);
    const int M = t.M;
    const GenPlan mg = generic_radices(M);
    a.gen.M = M;
    a.gen.mst = mg.nst;
    std::memcpy(a.gen.mradix, mg.radix, sizeof mg.radix);
    std::vector<float2> h((size_t)L + 2 * (size_t)M);
    for (int n = 0; n < L; ++n) h[(size_t)n] = make_float2((float)t.chirp[n].x, (float)t.chirp[n].y);
    for (int k = 0; k < M; ++k) {
        h[(size_t)L + k] = make_float2((float)t.bhat[k].x, (float)t.bhat[k].y);
        h[(size_t)L + M + k] = make_float2((float)t.tw[k].x, (float)t.tw[k].y);
    }
    const cudaError_t e = upload(h, &a.d_blu);
    if (e != cudaSuccess) return e;
    a.gen.chirp = a.d_blu;
    a.gen.bhat = a.d_blu + L;
    a.gen.twm = a.d_blu + L + M;
    return cudaSuccess;
}

// The FP64 plan of an axis: the radices of a.gen and FP64 tables (the axis
// table, and for a Bluestein length the FP64 chirp tables).
cudaError_t setup_axis64(Axis& a)
{
    a.gen64.L = a.gen.L;
    a.gen64.nst = a.gen.nst;
    std::memcpy(a.gen64.radix, a.gen.radix, sizeof a.gen.radix);
    cudaError_t e = upload64(forward_table64(a.L, a.L), &a.d_tw64);
    if (e != cudaSuccess || smooth2357(a.L)) return e;
    const int L = a.L;
    const BluesteinTables t = bluestein_tables(L);
    const int M = t.M;
    const GenPlan mg = generic_radices(M);
    a.gen64.M = M;
    a.gen64.mst = mg.nst;
    std::memcpy(a.gen64.mradix, mg.radix, sizeof mg.radix);
    std::vector<double2> h;
    h.reserve((size_t)L + 2 * (size_t)M);
    h.insert(h.end(), t.chirp.begin(), t.chirp.end());
    h.insert(h.end(), t.bhat.begin(), t.bhat.end());
    h.insert(h.end(), t.tw.begin(), t.tw.end());
    if ((e = upload64(h, &a.d_blu64)) != cudaSuccess) return e;
    a.gen64.chirp = a.d_blu64;
    a.gen64.bhat = a.d_blu64 + L;
    a.gen64.twm = a.d_blu64 + L + M;
    return cudaSuccess;
}

// The cluster-split column kernels of length L (at most two, in table order).
void find_split(int L, const SplitEntry* (&out)[2])
{
    int n = 0, k = 0;
    const SplitEntry* e = split_entries(&n);
    for (int i = 0; i < n && k < 2; ++i)
        if (e[i].L == L) out[k++] = &e[i];
}

const L2SplitEntry* find_l2split(int L)
{
    int n = 0;
    const L2SplitEntry* e = l2split_entries(&n);
    for (int i = 0; i < n; ++i)
        if (e[i].L == L) return &e[i];
    return nullptr;
}

const TmaSplitEntry* find_tma_split(int L)
{
    int n = 0;
    const TmaSplitEntry* e = tma_split_entries(&n);
    for (int i = 0; i < n; ++i)
        if (e[i].L == L) return &e[i];
    return nullptr;
}

// The TMA-fed cluster split runs a column pass when the residue views are
// TMA-addressable: an even axis stride (16-byte aligned residue bases and row
// strides), whole batch entries stacked at L * S, at least one tile of columns.
bool tma_split_ok(const Axis& a, const ColArgs& ca)
{
    return a.tsplit && ca.S % 2 == 0 && ca.Bs == (long long)a.L * ca.S && ca.C >= 16 &&
           ((uintptr_t)ca.data & 15) == 0;
}

cudaError_t run_l2split(const Axis& a, int dir, const ColArgs& ca, cudaStream_t s)
{
    SplitMaps maps{};
    const int C = a.l2split->C;
    const bool shift = ca.S & 1;  // odd stride: odd residues' rows start one value early, boxes 2 wider
    for (int r = 0; r < C; ++r) {
        const long long rs = r * ca.S;
        const int off = shift ? (int)(rs & 1) : 0;
        const cudaError_t e = encode_tensor_map_2d(&maps.map[r], ca.data + rs - off, 2ull * (ca.C + off),
                                                   (unsigned long long)ca.nb * (a.L / C), 8ull * C * ca.S,
                                                   shift ? 36u : 32u, 256);
        if (e != cudaSuccess) return e;
    }
    const ColL2SplitFn f = shift ? (dir < 0 ? a.l2split->fwd_shift : a.l2split->inv_shift)
                                 : (dir < 0 ? a.l2split->fwd : a.l2split->inv);
    return f(ca, maps, a.d_l2scratch, a.l2_ctas, s);
}

// The residue split applies to a column pass whose batch entries are stacked
// at L S, with at least 16 columns, and an even stride or the shifted form.
bool l2split_ok(const Axis& a, const ColArgs& ca)
{
    return a.l2split && a.d_l2scratch && (ca.S % 2 == 0 || a.l2split->fwd_shift) && ca.Bs == (long long)a.L * ca.S &&
           ca.C >= 16 && ((uintptr_t)ca.data & 15) == 0;
}

cudaError_t run_tma_split(const Axis& a, int dir, const ColArgs& ca, cudaStream_t s)
{
    SplitMaps maps{};
    const int C = a.tsplit->C;
    for (int r = 0; r < C; ++r) {
        const cudaError_t e = encode_tensor_map_2d(&maps.map[r], ca.data + r * ca.S, 2ull * ca.C,
                                                   (unsigned long long)ca.nb * (a.L / C), 8ull * C * ca.S, 32, 256);
        if (e != cudaSuccess) return e;
    }
    return dir < 0 ? a.tsplit->fwd(ca, maps, s) : a.tsplit->inv(ca, maps, s);
}

const TcEntry* find_tc(int L)
{
    int n = 0;
    const TcEntry* e = tc_entries(&n);
    for (int i = 0; i < n; ++i)
        if (e[i].L == L) return &e[i];
    return nullptr;
}

// Operand tables of the tensor-core radix-16 stages: the real 32 x 32 form of
// the 16-point DFT, G = [[Fr, -Fi], [Fi, Fr]] (F = exp(-+2 pi i n k / 16)),
// stored n-major, as 16-bit values: [fwd hi][fwd lo][inv hi][inv lo] with
// hi = bf16(G), lo = bf16(G - hi) computed from FP64 (split-BF16), or
// [fwd][0][inv][0] in FP16.
std::vector<uint16_t> tc_table(int dtype)
{
    std::vector<uint16_t> t(4 * 1024, 0);
    for (int dir = 0; dir < 2; ++dir) {
        const double sgn = dir == 0 ? -1.0 : 1.0;
        for (int n = 0; n < 32; ++n)
            for (int k = 0; k < 32; ++k) {
                double c, s;
                root_of_unity((long long)(n % 16) * (k % 16), 16, &c, &s);  // exp(+2 pi i nk/16)
                const double fr = c, fi = sgn * s;                          // F = fr + i fi
                double g;
                if (n < 16) g = (k < 16) ? fr : -fi;
                else g = (k < 16) ? fi : fr;
                uint16_t* hi = &t[(size_t)dir * 2048 + (size_t)n * 32 + k];
                uint16_t* lo = hi + 1024;
                if (dtype == FFT3D_F32_TC_BF16X3) {
                    const __nv_bfloat16 h = __float2bfloat16_rn((float)g);
                    const __nv_bfloat16 l = __float2bfloat16_rn((float)(g - (double)__bfloat162float(h)));
                    *hi = __bfloat16_as_ushort(h);
                    *lo = __bfloat16_as_ushort(l);
                } else {
                    *hi = __half_as_ushort(__float2half_rn((float)g));
                    *lo = 0;
                }
            }
    }
    return t;
}

}  // namespace

enum PassId { PASS_ROW_R2C = 0, PASS_N1_FWD, PASS_N0_FWD, PASS_N0_INV, PASS_N1_INV, PASS_ROW_C2R, PASS_SWAP01,
              PASS_PLANE_FWD, PASS_PLANE_INV, PASS_COUNT };
const char* const kPassNames[PASS_COUNT] = {"row_r2c",    "col_n1_fwd", "col_n0_fwd", "col_n0_inv", "col_n1_inv",
                                            "row_c2r",    "swap01",     "plane_fwd",  "plane_inv"};

struct ProfRecord {
    int pass;
    cudaEvent_t a, b;
};

struct fft3d_plan_s {
    int n0 = 0, n1 = 0, n2 = 0, H = 0, batch = 0, dtype = 0, flags = 0;
    long long N = 0, M = 0, P = 0;
    int device = 0;
    Axis ax0, ax1, ax2;  // ax2: the row transform, length n2/2 (even n2) or n2 (odd n2)
    float2* d_twpack = nullptr;
    double2* d_twpack64 = nullptr;  // FFT3D_F64 plans
    int* d_status = nullptr;
    const PlaneEntry* plane = nullptr;  // fused n2+n1 kernel, when one fits this shape
    const CPlaneEntry* cplane = nullptr;  // cluster (distributed shared memory) n2+n1 kernel
    uint16_t* d_tcg = nullptr;          // tensor-core DFT operand table (TC dtypes)
    int* d_counters = nullptr;          // per-plane completion counters + work ticket of the fused kernel
    float2* d_ring = nullptr;           // inverse fused kernel: L2-resident ring of n1-transformed planes
    int ring_planes = 0;
    double* d_energy = nullptr;         // scratch of fft3d_energy (block partials)
    size_t energy_doubles = 0;
    // kernel shape choices (autotuner): columns per CTA of the n0 / n1 column
    // kernels, rows per CTA of the row kernels (0: compiled default), and
    // whether the n0 pass may use the TMA kernel
    int choice_w0 = 0, choice_w1 = 0, choice_rows = 0, choice_tma = 1, choice_tma1 = 1;
    float2* d_l2scratch = nullptr;  // the residue-split column kernels' scratch (both axes)
    void* workspace = nullptr;
    std::string desc;
    bool profiling = false;
    std::vector<ProfRecord> prof;  // event pairs, reused across reads
    size_t prof_used = 0;
    // tensor maps of recent column-pass operands, keyed by (base, stride)
    struct MapCache {
        const void* base = nullptr;
        long long S = 0, C = 0, nb = 0;
        bool pair = false;
        CUtensorMap map;
    } maps[8];
    int next_map = 0;
    std::mutex maps_mutex;  // guards maps / next_map (a plan may serve several host threads)
};

namespace {

cudaError_t upload(const std::vector<float2>& h, float2** d)
{
    cudaError_t e = cudaMalloc((void**)d, h.size() * sizeof(float2));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*d, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice);
}

void free_plan(fft3d_plan_s* p)
{
    if (!p) return;
    for (ProfRecord& r : p->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (Axis* a : {&p->ax0, &p->ax1, &p->ax2}) {
        cudaFree(a->d_tw);
        cudaFree(a->d_blu);
        cudaFree(a->d_tw64);
        cudaFree(a->d_blu64);
    }
    cudaFree(p->d_l2scratch);
    cudaFree(p->d_twpack64);
    cudaFree(p->d_twpack);
    cudaFree(p->d_status);
    cudaFree(p->d_counters);
    cudaFree(p->d_ring);
    cudaFree(p->d_energy);
    cudaFree(p->d_tcg);
    delete p;
}

// Brackets one launch with events when the plan is profiling.
// One pass: an NVTX range named for the pass around its launch (host side,
// seen by a tracing tool), and CUDA events around it while profiling is on.
struct ProfScope {
    fft3d_plan_s* p;
    ProfRecord* r = nullptr;
    cudaStream_t s;
    ProfScope(fft3d_plan_s* plan, int pass, cudaStream_t stream) : p(plan), s(stream)
    {
        nvtxRangePushA(kPassNames[pass]);
        if (!p->profiling) return;
        if (p->prof_used == p->prof.size()) {
            ProfRecord nr{pass, nullptr, nullptr};
            if (cudaEventCreate(&nr.a) != cudaSuccess || cudaEventCreate(&nr.b) != cudaSuccess) return;
            p->prof.push_back(nr);
        }
        r = &p->prof[p->prof_used++];
        r->pass = pass;
        cudaEventRecord(r->a, s);
    }
    ~ProfScope()
    {
        if (r) cudaEventRecord(r->b, s);
        nvtxRangePop();
    }
};

bool uses_generic(const fft3d_plan_s* p, const Axis& a, bool row)
{
    if (p->flags & FFT3D_FLAG_GENERIC) return true;
    if (!a.spec) return true;
    return row ? (a.spec->r2c == nullptr) : false;
}

// The TMA column kernel needs a 2D tensor view: batch entries stacked as rows
// (Bs == L*S) and at least one tile of columns; an even S gives a row stride
// that is a multiple of 16 bytes, an odd S is handled by the row-pair view
// (needs an even L).  Returns 0 (no TMA), 1 (rows) or 2 (row pairs).
int tma_mode(const fft3d_plan_s* p, const Axis& a, long long S, long long C, long long Bs)
{
    if (p->flags & FFT3D_FLAG_GENERIC) return 0;
    if (!a.spec || !a.spec->tma_W) return 0;
    if (Bs != (long long)a.L * S || C < a.spec->tma_W) return 0;
    if (S % 2 == 0) return 1;
    return (a.L % 2 == 0 && a.spec->tma_pair_fwd) ? 2 : 0;
}

bool tma_ok(const fft3d_plan_s* p, const Axis& a, long long S, long long C, long long Bs)
{
    return tma_mode(p, a, S, C, Bs) != 0;
}

// The tensor map of a column-pass operand, copied into *out (the cache is
// shared by every host thread that uses the plan, so it is read and written
// under the plan's lock, and the caller launches with its own copy).
bool tensor_map(fft3d_plan_s* p, const Axis& a, const ColArgs& ca, bool pair, CUtensorMap* out)
{
    std::lock_guard<std::mutex> lock(p->maps_mutex);
    for (auto& m : p->maps)
        if (m.base == ca.data && m.S == ca.S && m.C == ca.C && m.nb == ca.nb && m.pair == pair) {
            *out = m.map;
            return true;
        }
    auto& m = p->maps[p->next_map];
    p->next_map = (p->next_map + 1) % 8;
    if (col_tensor_map_host(&m.map, ca, a.L, a.spec->tma_W, pair) != cudaSuccess) {
        m.base = nullptr;
        return false;
    }
    m.base = ca.data;
    m.S = ca.S;
    m.C = ca.C;
    m.nb = ca.nb;
    m.pair = pair;
    *out = m.map;
    return true;
}

// The cluster-split kernel the plan's choice selects for this column axis, or nullptr.
const SplitEntry* split_choice(const fft3d_plan_s* p, const Axis& a)
{
    const int form = (&a == &p->ax0) ? p->choice_tma : p->choice_tma1;
    return (form == 2 || form == 3) ? a.split[form - 2] : nullptr;
}

// One column pass with full control of the arguments (destination, mask, scale).
cudaError_t launch_col_args(fft3d_plan_s* p, const Axis& a, int dir, const ColArgs& ca, cudaStream_t s)
{
    if (a.L <= 1) {  // length-1 axis: the transform is the identity (apart from scale / mask / destination)
        if (!ca.dst && ca.scale == 1.0f) return cudaSuccess;
    }
    if (ca.nb2 > 1 && (uses_generic(p, a, false) || a.tc || !a.spec)) {
        // an outer batch on a path without it: one pass per group
        for (long long b2 = 0; b2 < ca.nb2; ++b2) {
            ColArgs c = ca;
            c.data += b2 * ca.Bs2;
            if (c.dst) c.dst += b2 * ca.Bs2;
            c.nb2 = 1;
            c.Bs2 = 0;
            const cudaError_t e = launch_col_args(p, a, dir, c, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (a.tc) {  // tensor-core radix-16 stages
        if (p->dtype == FFT3D_F32_TC_BF16X3)
            return dir < 0 ? a.tc->bf16_fwd(ca, p->d_tcg, s) : a.tc->bf16_inv(ca, p->d_tcg, s);
        return dir < 0 ? a.tc->f16_fwd(ca, p->d_tcg, s) : a.tc->f16_inv(ca, p->d_tcg, s);
    }
    if (uses_generic(p, a, false)) return generic_col(ca, a.gen, dir, s);
    const bool n0axis = (&a == &p->ax0);
    if (ca.nb2 > 1) {  // an outer batch: the plain column kernel is the form that takes it
        const int w = n0axis ? p->choice_w0 : p->choice_w1;
        return dir < 0 ? a.spec->col_fwd(ca, w, s) : a.spec->col_inv(ca, w, s);
    }
    const int form = n0axis ? p->choice_tma : p->choice_tma1;
    if (form == 4 && tma_split_ok(a, ca)) return run_tma_split(a, dir, ca, s);  // TMA-fed cluster split
    if (form == 5 && l2split_ok(a, ca)) return run_l2split(a, dir, ca, s);     // residue split through L2
    if ((form == 2 || form == 3) && a.split[form - 2]) {  // cluster-split kernel
        const SplitEntry* se = a.split[form - 2];
        return dir < 0 ? se->fwd(ca, 0, s) : se->inv(ca, 0, s);
    }
    const int mode = tma_mode(p, a, ca.S, ca.C, ca.Bs);
    if (form == 6 && mode == 2 && a.spec->tma_pair2_fwd) {  // row pairs, two columns per thread
        CUtensorMap m;
        if (tensor_map(p, a, ca, true, &m)) return dir < 0 ? a.spec->tma_pair2_fwd(ca, m, s) : a.spec->tma_pair2_inv(ca, m, s);
    }
    if ((form == 1 || form == 6) && mode) {
        CUtensorMap m;
        if (tensor_map(p, a, ca, mode == 2, &m)) {
            if (mode == 2) return dir < 0 ? a.spec->tma_pair_fwd(ca, m, s) : a.spec->tma_pair_inv(ca, m, s);
            return dir < 0 ? a.spec->tma_fwd(ca, m, s) : a.spec->tma_inv(ca, m, s);
        }
    }
    const int w = n0axis ? p->choice_w0 : p->choice_w1;
    return dir < 0 ? a.spec->col_fwd(ca, w, s) : a.spec->col_inv(ca, w, s);
}

// dst: the result goes there (same layout) and data is only read; nullptr: in place
cudaError_t run_col(fft3d_plan_s* p, const Axis& a, int dir, float2* data, long long S, long long C,
                    long long nb, long long Bs, cudaStream_t s, float2* dst = nullptr)
{
    if (a.L <= 1) return cudaSuccess;
    const bool n0axis = (&a == &p->ax0);
    ProfScope ps(p, n0axis ? (dir < 0 ? PASS_N0_FWD : PASS_N0_INV) : (dir < 0 ? PASS_N1_FWD : PASS_N1_INV), s);
    ColArgs ca{data, S, C, nb, Bs, a.d_tw, 1.0f, p->d_status, dst, 0};
    return launch_col_args(p, a, dir, ca, s);
}

cudaError_t run_row(fft3d_plan_s* p, int dir, const void* in, void* out, cudaStream_t s)
{
    ProfScope ps(p, dir < 0 ? PASS_ROW_R2C : PASS_ROW_C2R, s);
    // real rows: n2 floats, or 2H floats in the padded (in-place capable) layout
    const bool padded = p->flags & FFT3D_FLAG_PADDED_REAL;
    if (p->n2 & 1) {  // odd n2: full-length complex row transform, stride in floats
        RowArgs ra{in, out, (long long)p->batch * p->n0 * p->n1, p->ax2.d_tw, p->d_twpack,
                   padded ? 2 * p->H : (long long)p->n2};
        return generic_row_odd(ra, p->ax2.gen, dir, s);
    }
    const long long rs = padded ? p->H : p->n2 / 2;
    RowArgs ra{in, out, (long long)p->batch * p->n0 * p->n1, p->ax2.d_tw, p->d_twpack, rs};
    if (uses_generic(p, p->ax2, true)) return generic_row(ra, p->ax2.gen, dir, s);
    return dir < 0 ? p->ax2.spec->r2c(ra, p->choice_rows, s) : p->ax2.spec->c2r(ra, p->choice_rows, s);
}

std::string axis_desc(const fft3d_plan_s* p, const Axis& a, bool row)
{
    char b[96];
    if (a.L <= 1) return "skip";
    if (!row && a.tc) {
        std::snprintf(b, sizeof b, "L=%d E=16 cols/CTA=%d tensor-core radix-16 %s", a.L, a.tc->W,
                      p->dtype == FFT3D_F32_TC_BF16X3 ? "split-bf16x3" : "fp16");
        return b;
    }
    if (uses_generic(p, a, row)) {
        if (a.gen.M)
            std::snprintf(b, sizeof b, "generic L=%d bluestein M=%d", a.L, a.gen.M);
        else
            std::snprintf(b, sizeof b, "generic L=%d", a.L);
    } else if (row) {
        const int rr = (p->choice_rows > 0 && p->choice_rows <= a.spec->row_rows && a.spec->row_warp)
                           ? p->choice_rows
                           : a.spec->row_rows;
        std::snprintf(b, sizeof b, "L=%d E=%d rows/CTA=%d %s", a.L, a.spec->row_E, rr,
                      a.spec->row_warp ? "warp" : "smem");
    } else if (((&a == &p->ax0) ? p->choice_tma : p->choice_tma1) == 6 && a.spec->tma_pair2_fwd &&
               (&a == &p->ax0 ? tma_mode(p, a, p->P, p->P, p->M) : tma_mode(p, a, p->H, p->H, (long long)p->n1 * p->H)) == 2) {
        std::snprintf(b, sizeof b, "L=%d E=%d cols/CTA=%d tma-row-pairs 2 cols/thread", a.L, a.spec->tma_pair_E,
                      a.spec->tma_W);
    } else if (((&a == &p->ax0) ? p->choice_tma : p->choice_tma1) == 5 && a.l2split) {
        std::snprintf(b, sizeof b, "L=%d E=32 cols/CTA=16 tma-residue-split C=%d via L2", a.L, a.l2split->C);
    } else if (((&a == &p->ax0) ? p->choice_tma : p->choice_tma1) == 4 && a.tsplit &&
               (&a == &p->ax0 ? p->P % 2 == 0 && p->P >= 16 : p->H % 2 == 0 && p->H >= 16)) {
        std::snprintf(b, sizeof b, "L=%d E=32 cols/CTA=16 tma-cluster-split C=%d", a.L, a.tsplit->C);
    } else if (const SplitEntry* se = split_choice(p, a)) {
        std::snprintf(b, sizeof b, "L=%d E=%d cols/CTA=%d cluster-split C=%d", a.L, se->E, se->W, se->C);
    } else if (const int mode = (&a == &p->ax0) ? (p->choice_tma == 1 ? tma_mode(p, a, p->P, p->P, p->M) : 0)
                                                : (p->choice_tma1 == 1 ? tma_mode(p, a, p->H, p->H, (long long)p->n1 * p->H)
                                                                       : 0)) {
        std::snprintf(b, sizeof b, "L=%d E=%d cols/CTA=%d %s", a.L, mode == 2 ? a.spec->tma_pair_E : a.spec->tma_E,
                      a.spec->tma_W, mode == 2 ? "tma-row-pairs" : "tma");
    } else {
        const int w = (&a == &p->ax0) ? p->choice_w0 : p->choice_w1;
        std::snprintf(b, sizeof b, "L=%d E=%d cols/CTA=%d", a.L, a.spec->col_E,
                      (w > 0 && w <= a.spec->col_W) ? w : a.spec->col_W);
    }
    return b;
}

// The fused plane pass (rows + n1 columns of every plane in one launch).
cudaError_t run_plane(fft3d_plan_s* p, int dir, const void* in, void* out, cudaStream_t s)
{
    ProfScope ps(p, dir < 0 ? PASS_PLANE_FWD : PASS_PLANE_INV, s);
    const long long planes = (long long)p->batch * p->n0;
    cudaError_t e = cudaMemsetAsync(p->d_counters, 0, (size_t)(((planes + 1) & ~1LL) + 2) * sizeof(int), s);
    if (e != cudaSuccess) return e;
    PlaneArgs a;
    a.in = in;
    a.out = out;
    a.planes = planes;
    a.H = p->H;
    a.tw_row = p->ax2.d_tw;
    a.twpack = p->d_twpack;
    a.tw_col = p->ax1.d_tw;
    a.counters = p->d_counters;
    a.ring = p->d_ring;
    a.ring_planes = p->ring_planes;
    a.status = p->d_status;
    a.lag = 2;
    const bool test_skip = p->flags & FFT3D_FLAG_TEST_SKIP_ARRIVAL;
    a.wait_limit = test_skip ? 4000u : 20000000u;  // ~1 ms in the test hook, seconds otherwise
    a.skip_plane = test_skip ? 0 : -1;
    return dir < 0 ? p->plane->fwd(a, s) : p->plane->inv(a, s);
}

// The cluster plane kernel of shape (n2/2 = LR, n1 = LC) with cluster size C
// (C = 0: the shape's default, the first listed), or nullptr.
const CPlaneEntry* cplane_for(int LR, int LC, int C)
{
    int nc = 0;
    const CPlaneEntry* ce = cplane_entries(&nc);
    for (int i = 0; i < nc; ++i)
        if (ce[i].LR == LR && ce[i].LC == LC && (C == 0 || ce[i].C == C)) return &ce[i];
    return nullptr;
}

// The plan may replace its row and n1 passes by a cluster plane pass.
bool cplane_allowed(const fft3d_plan_s* p)
{
    return p->dtype == FFT3D_F32 && !p->plane && (p->n2 % 2 == 0) &&
           !(p->flags & (FFT3D_FLAG_THREE_PASS | FFT3D_FLAG_GENERIC | FFT3D_FLAG_EXPLICIT_TRANSPOSE |
                         FFT3D_FLAG_FUSED_PLANE | FFT3D_FLAG_PADDED_REAL));
}

// The cluster plane pass (rows + n1 columns of every plane, one cluster per plane).
cudaError_t run_cplane(fft3d_plan_s* p, int dir, const void* in, void* out, cudaStream_t s)
{
    ProfScope ps(p, dir < 0 ? PASS_PLANE_FWD : PASS_PLANE_INV, s);
    CPlaneArgs a;
    a.in = in;
    a.out = out;
    a.planes = (long long)p->batch * p->n0;
    a.tw_row = p->ax2.d_tw;
    a.twpack = p->d_twpack;
    a.tw_col = p->ax1.d_tw;
    a.status = p->d_status;
    return dir < 0 ? p->cplane->fwd(a, s) : p->cplane->inv(a, s);
}

cudaError_t run_swap(fft3d_plan_s* p, const float2* in, float2* out, long long a0, long long a1, cudaStream_t s)
{
    ProfScope ps(p, PASS_SWAP01, s);
    return launch_swap01(in, out, p->batch, a0, a1, p->H, s);
}

std::string describe_plan(const fft3d_plan_s* p)
{
    const int flags = p->flags;
    std::string d = "rows[" + axis_desc(p, p->ax2, true) + "] n1[" + axis_desc(p, p->ax1, false) + "] n0[" +
                    axis_desc(p, p->ax0, false) + "]";
    if (p->cplane) {
        char b[128];
        std::snprintf(b, sizeof b, "cluster-plane[%d CTAs x %d rows, %d threads]", p->cplane->C,
                      p->cplane->LC / p->cplane->C, p->cplane->NT);
        d = std::string(b) + " n0[" + axis_desc(p, p->ax0, false) + "]";
    }
    if (p->plane) {
        char b[128];
        std::snprintf(b, sizeof b, "plane[fused rows E=%d + n1 E=%d, %d threads]", p->plane->ER, p->plane->EC,
                      p->plane->NT);
        d = std::string(b) + " n0[" + axis_desc(p, p->ax0, false) + "]";
    }
    if (flags & FFT3D_FLAG_EXPLICIT_TRANSPOSE)
        d += (flags & FFT3D_FLAG_TRANSPOSE_BACK) ? " explicit-transpose+back" : " explicit-transpose";
    if (p->dtype == FFT3D_F64) d = "fp64 " + d;
    return d;
}

// Bytes of the real side: n2 floats per row, or 2H in the padded layout.
size_t real_bytes(const fft3d_plan_s* p)
{
    const size_t row = (p->flags & FFT3D_FLAG_PADDED_REAL) ? 2 * (size_t)p->H : (size_t)p->n2;
    return (size_t)p->batch * p->n0 * p->n1 * row * sizeof(float);
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb)
{
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
}

}  // namespace

extern "C" {

const char* fft3d_error_string(int status)
{
    switch (status) {
    case FFT3D_OK: return "ok";
    case FFT3D_ERR_INVALID_ARG: return "invalid argument";
    case FFT3D_ERR_UNSUPPORTED_SIZE: return "unsupported size (n0, n1 and n2/2 (n2 for odd n2) must be <= 4096) or form not offered at this size";
    case FFT3D_ERR_MISALIGNED: return "data pointer not 16-byte aligned";
    case FFT3D_ERR_ALLOC: return "device allocation failed";
    case FFT3D_ERR_CUDA: return "CUDA error";
    case FFT3D_ERR_TIMEOUT: return "device-side wait timed out";
    case FFT3D_ERR_NO_WORKSPACE: return "plan needs caller workspace (fft3d_set_workspace)";
    default: return "unknown status";
    }
}

int fft3d_last_error(void) { return g_last_error; }

fft3d_handle fft3d_plan_variant(int n0, int n1, int n2, int dtype, int batch, int flags)
{
    if (dtype != FFT3D_F64) flags |= forced_flags();
    if (n0 < 1 || n1 < 1 || n2 < 2 || batch < 1 || dtype < 0 || dtype > FFT3D_F64 ||
        (dtype == FFT3D_F64 && flags != 0) ||
        (flags & ~(FFT3D_FLAG_EXPLICIT_TRANSPOSE | FFT3D_FLAG_TRANSPOSE_BACK | FFT3D_FLAG_THREE_PASS |
                   FFT3D_FLAG_GENERIC | FFT3D_FLAG_TEST_SKIP_ARRIVAL | FFT3D_FLAG_FUSED_PLANE |
                   FFT3D_FLAG_CLUSTER_PLANE | FFT3D_FLAG_PADDED_REAL | FFT3D_FLAG_PRESERVE_INPUT)) ||
        ((flags & FFT3D_FLAG_TRANSPOSE_BACK) && !(flags & FFT3D_FLAG_EXPLICIT_TRANSPOSE)) ||
        // the padded layout and the input-preserving inverse run the transpose-free pass sequence
        ((flags & (FFT3D_FLAG_PADDED_REAL | FFT3D_FLAG_PRESERVE_INPUT)) &&
         (flags & (FFT3D_FLAG_EXPLICIT_TRANSPOSE | FFT3D_FLAG_FUSED_PLANE)))) {
        fail(FFT3D_ERR_INVALID_ARG);
        return nullptr;
    }
    // the row transform has length n2/2 (even n2, half-length packing) or n2 (odd n2)
    const int row_len = (n2 & 1) ? n2 : n2 / 2;
    if (n0 < 1 || n1 < 1 || row_len < 1 || n0 > kMaxAxis || n1 > kMaxAxis || row_len > kMaxAxis) {
        fail(FFT3D_ERR_UNSUPPORTED_SIZE);
        return nullptr;
    }
    // FP64: a Bluestein line of M = 8192 double2 points (two buffers) does not fit one CTA
    if (dtype == FFT3D_F64)
        for (int L : {n0, n1, row_len})
            if (!smooth2357(L) && L > kMaxAxis / 2) {
                fail(FFT3D_ERR_UNSUPPORTED_SIZE);
                return nullptr;
            }
    if (dtype != FFT3D_F32 && (flags & (FFT3D_FLAG_EXPLICIT_TRANSPOSE | FFT3D_FLAG_GENERIC | FFT3D_FLAG_FUSED_PLANE |
                                        FFT3D_FLAG_CLUSTER_PLANE))) {
        fail(FFT3D_ERR_INVALID_ARG);  // the tensor-core forms use the plain transpose-free pass sequence
        return nullptr;
    }
    fft3d_plan_s* p = new (std::nothrow) fft3d_plan_s();
    if (!p) {
        fail(FFT3D_ERR_ALLOC);
        return nullptr;
    }
    p->n0 = n0;
    p->n1 = n1;
    p->n2 = n2;
    p->H = n2 / 2 + 1;
    p->batch = batch;
    p->dtype = dtype;
    p->flags = flags;
    p->N = (long long)n0 * n1 * n2;
    p->P = (long long)n1 * p->H;
    p->M = (long long)n0 * p->P;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        fail(FFT3D_ERR_CUDA);
        return nullptr;
    }
    Axis* axes[3] = {&p->ax0, &p->ax1, &p->ax2};
    const int lens[3] = {n0, n1, row_len};
    for (int i = 0; i < 3; ++i) {
        Axis& a = *axes[i];
        a.L = lens[i];
        // odd rows and the FP64 path: the runtime-length kernels
        a.spec = ((i == 2 && (n2 & 1)) || dtype == FFT3D_F64) ? nullptr : find_len(a.L);
        a.tc = (is_tc_dtype(dtype) && i < 2) ? find_tc(a.L) : nullptr;
        if (a.spec && i < 2) {
            find_split(a.L, a.split);
            a.tsplit = find_tma_split(a.L);
        }
        // the residue split of a column pass: an axis stride of at least 16
        // columns, even, or odd where the length has the shifted form
        const long long stride = i == 0 ? p->P : p->H;
        if (a.spec && i < 2 && stride >= 16 && dtype == FFT3D_F32 && !(flags & FFT3D_FLAG_EXPLICIT_TRANSPOSE))
            if (const L2SplitEntry* le = find_l2split(a.L))
                if (stride % 2 == 0 || le->fwd_shift) {
                    a.l2split = le;
                    a.l2_ctas = le->ctas();
                }
        a.gen = generic_radices(a.L);
        if (upload(forward_table(a.L, a.L), &a.d_tw) != cudaSuccess ||
            (!smooth2357(a.L) && setup_bluestein(a) != cudaSuccess) ||
            (dtype == FFT3D_F64 && setup_axis64(a) != cudaSuccess)) {
            free_plan(p);
            fail(FFT3D_ERR_ALLOC);
            return nullptr;
        }
    }
    {
        // the residue split's scratch: one region per resident CTA, shared by
        // both axes (a plan's passes run one after another on its stream)
        size_t bytes = 0;
        for (Axis* a : {&p->ax0, &p->ax1})
            if (a->l2split && a->l2_ctas > 0)
                bytes = std::max(bytes, a->l2split->scratch_values(a->l2_ctas) * sizeof(float2));
        float2* scratch = nullptr;
        if (bytes && cudaMalloc((void**)&scratch, bytes) == cudaSuccess) p->d_l2scratch = scratch;
        cudaGetLastError();  // a failed allocation only leaves the form out
        for (Axis* a : {&p->ax0, &p->ax1}) {
            if (!p->d_l2scratch || a->l2_ctas <= 0) a->l2split = nullptr;
            a->d_l2scratch = a->l2split ? p->d_l2scratch : nullptr;
        }
    }
    // default n0-pass kernel: the plain kernel for long n0 axes, whose rows lie
    // megabytes apart (GB300: n0 = 1024, 16-wide 4.2 TB/s vs TMA 8-wide 2.9;
    // n0 = 1536, 8-wide 2.9 vs 2.5; n0 = 2048, 8-wide 3.0 vs TMA 4-wide 1.3),
    // n0 = 768 (8-wide TMA tiles 1.18 ms vs plain 16-wide 1.07 at 768^3) and
    // n0 <= 64 (64^3 x 4 fields: 6.8 vs 7.5 us); the TMA kernel from 96 to
    // 640 (128^3 x 4: 15.5 vs 18.5 us, 192^3 x 4: 41 vs 53, 384^3: 96 vs 122,
    // 640^3: 0.56 vs 0.69 ms)
    if (p->ax0.spec && p->ax0.spec->tma_W && (p->ax0.L <= 64 || p->ax0.L >= 768)) p->choice_tma = 0;
    // n0 = 1024, 1536, 2048: the residue split through L2 where it applies
    // (GB300, n0 pass: 1.94 vs 2.05 ms at 1024^3, 6.5-7.3 vs 8.4-8.5 ms at
    // 1536 x 1024 x 2048, 18.9-19.6 vs 22.3-22.5 ms at 2048^3)
    if (p->ax0.l2split) p->choice_tma = 5;
    if (is_tc_dtype(dtype)) {
        if (!p->ax0.tc && !p->ax1.tc) {  // no axis with a tensor-core kernel: the form does not exist here
            free_plan(p);
            fail(FFT3D_ERR_UNSUPPORTED_SIZE);
            return nullptr;
        }
        const std::vector<uint16_t> t = tc_table(dtype);
        if (cudaMalloc((void**)&p->d_tcg, t.size() * sizeof(uint16_t)) != cudaSuccess ||
            cudaMemcpy(p->d_tcg, t.data(), t.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess) {
            free_plan(p);
            fail(FFT3D_ERR_ALLOC);
            return nullptr;
        }
    }
    if (upload(forward_table(n2, n2 / 2 + 1), &p->d_twpack) != cudaSuccess ||
        (dtype == FFT3D_F64 && upload64(forward_table64(n2, n2 / 2 + 1), &p->d_twpack64) != cudaSuccess) ||
        cudaMalloc((void**)&p->d_status, sizeof(int)) != cudaSuccess ||
        cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess) {
        free_plan(p);
        fail(FFT3D_ERR_ALLOC);
        return nullptr;
    }
    if ((flags & FFT3D_FLAG_FUSED_PLANE) &&
        !(flags & (FFT3D_FLAG_THREE_PASS | FFT3D_FLAG_GENERIC | FFT3D_FLAG_EXPLICIT_TRANSPOSE))) {
        int np = 0;
        const PlaneEntry* pe = plane_entries(&np);
        for (int i = 0; i < np; ++i)
            if (n2 % 2 == 0 && pe[i].LR == n2 / 2 && pe[i].LC == n1) p->plane = &pe[i];
        // per-plane counters, then an 8-byte work ticket (kept 8-byte aligned)
        const size_t ncount = (((size_t)batch * n0 + 1) & ~(size_t)1) + 2;
        if (p->plane && cudaMalloc((void**)&p->d_counters, ncount * sizeof(int)) != cudaSuccess) {
            free_plan(p);
            fail(FFT3D_ERR_ALLOC);
            return nullptr;
        }
        // Inverse ring: as many planes as can be in flight (bounded by the item
        // lag the kernel derives, well under this) so the clobbered spectrum
        // is never written back to DRAM.  At most 64 MiB.
        if (p->plane) {
            const size_t plane_bytes = (size_t)n1 * (n2 / 2 + 1) * sizeof(float2);
            int rp = (int)((64u << 20) / plane_bytes);
            if (rp > 32) rp = 32;
            if (rp >= 16 && (long long)rp < (long long)batch * n0) {
                if (cudaMalloc((void**)&p->d_ring, (size_t)rp * plane_bytes) != cudaSuccess) {
                    free_plan(p);
                    fail(FFT3D_ERR_ALLOC);
                    return nullptr;
                }
                p->ring_planes = rp;
            }
        }
    }
    if ((flags & FFT3D_FLAG_CLUSTER_PLANE) && cplane_allowed(p)) p->cplane = cplane_for(n2 / 2, n1, 0);
    {
        // energy scratch for nbins up to the largest shell of the shape
        const double kmax = std::sqrt((double)(n0 / 2) * (n0 / 2) + (double)(n1 / 2) * (n1 / 2) +
                                      (double)(n2 / 2) * (n2 / 2));
        const int nb = (int)kmax + 2;
        p->energy_doubles = energy_scratch_doubles(batch, (long long)n0 * n1, nb);
        if (cudaMalloc((void**)&p->d_energy, p->energy_doubles * sizeof(double)) != cudaSuccess) {
            free_plan(p);
            fail(FFT3D_ERR_ALLOC);
            return nullptr;
        }
    }
    p->desc = describe_plan(p);
    if (log_enabled())
        std::fprintf(stderr, "fft3d: plan %dx%dx%d batch=%d dtype=%d flags=0x%x: %s\n", n0, n1, n2, batch, dtype, flags,
                     p->desc.c_str());
    return p;
}

fft3d_handle fft3d_plan(int n0, int n1, int n2, int dtype, int batch)
{
    return fft3d_plan_variant(n0, n1, n2, dtype, batch, 0);
}

void fft3d_destroy(fft3d_handle p)
{
    if (!p) return;
    cudaDeviceSynchronize();
    free_plan(p);
}

size_t fft3d_workspace_bytes(fft3d_handle p)
{
    if (!p) return 0;
    if (p->flags & (FFT3D_FLAG_EXPLICIT_TRANSPOSE | FFT3D_FLAG_PRESERVE_INPUT))
        return (size_t)p->batch * (size_t)p->M * sizeof(float2);
    return 0;
}

int fft3d_set_workspace(fft3d_handle p, void* dev_ptr)
{
    if (!p) return fail(FFT3D_ERR_INVALID_ARG);
    if (dev_ptr && ((uintptr_t)dev_ptr & 255)) return fail(FFT3D_ERR_MISALIGNED);
    p->workspace = dev_ptr;
    return FFT3D_OK;
}

int fft3d_describe(fft3d_handle p, char* text, int len)
{
    if (!p || !text || len < 1) return fail(FFT3D_ERR_INVALID_ARG);
    std::snprintf(text, (size_t)len, "%dx%dx%d batch=%d %s", p->n0, p->n1, p->n2, p->batch, describe_plan(p).c_str());
    return FFT3D_OK;
}

int fft3d_launches_per_call(fft3d_handle p, int dir)
{
    if (!p) return fail(FFT3D_ERR_INVALID_ARG);
    (void)dir;
    if (p->plane || p->cplane) return 1 + (p->n0 > 1);
    int n = 1 + (p->n1 > 1) + (p->n0 > 1);
    if (p->flags & FFT3D_FLAG_EXPLICIT_TRANSPOSE) n += (p->flags & FFT3D_FLAG_TRANSPOSE_BACK) ? 2 : 1;
    return n;
}

int fft3d_query_device_status(fft3d_handle p, void* stream)
{
    if (!p) return fail(FFT3D_ERR_INVALID_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    int h = 0;
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
    if (cudaMemcpy(&h, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess)
        return fail(FFT3D_ERR_CUDA);
    return h == 0 ? FFT3D_OK : fail(FFT3D_ERR_TIMEOUT);
}

int fft3d_r2c(fft3d_handle p, const float* in, void* out, void* stream)
{
    if (!p || !in || !out || p->dtype == FFT3D_F64) return fail(FFT3D_ERR_INVALID_ARG);
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return fail(FFT3D_ERR_MISALIGNED);
    const size_t in_bytes = real_bytes(p);
    const size_t out_bytes = (size_t)p->batch * p->M * sizeof(float2);
    const bool in_place = (p->flags & FFT3D_FLAG_PADDED_REAL) && (const void*)in == out;
    if (!in_place && overlaps(in, in_bytes, out, out_bytes)) return fail(FFT3D_ERR_INVALID_ARG);
    const bool xpose = p->flags & FFT3D_FLAG_EXPLICIT_TRANSPOSE;
    if (xpose && !p->workspace) return fail(FFT3D_ERR_NO_WORKSPACE);
    cudaStream_t s = (cudaStream_t)stream;
    const long long H = p->H, n0 = p->n0, n1 = p->n1, B = p->batch;
    float2* o = (float2*)out;
    cudaError_t e;
    if (!xpose && p->cplane) {
        if (run_cplane(p, -1, in, o, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_col(p, p->ax0, -1, o, p->P, p->P, B, p->M, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        return FFT3D_OK;
    }
    if (!xpose && p->plane) {
        if (run_plane(p, -1, in, o, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_col(p, p->ax0, -1, o, p->P, p->P, B, p->M, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        return FFT3D_OK;
    }
    if (!xpose) {
        if ((e = run_row(p, -1, in, o, s)) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if ((e = run_col(p, p->ax1, -1, o, H, H, B * n0, n1 * H, s)) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if ((e = run_col(p, p->ax0, -1, o, p->P, p->P, B, p->M, s)) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        return FFT3D_OK;
    }
    float2* w = (float2*)p->workspace;
    if (!(p->flags & FFT3D_FLAG_TRANSPOSE_BACK)) {
        // plane passes into the workspace, transpose into out, n0 pass on out
        // (now the middle axis: element (k1, j0, k2) at (k1*n0 + j0)*H + k2)
        if (run_row(p, -1, in, w, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_col(p, p->ax1, -1, w, H, H, B * n0, n1 * H, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_swap(p, w, o, n0, n1, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_col(p, p->ax0, -1, o, H, H, B * n1, n0 * H, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
    } else {
        if (run_row(p, -1, in, o, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_col(p, p->ax1, -1, o, H, H, B * n0, n1 * H, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_swap(p, o, w, n0, n1, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_col(p, p->ax0, -1, w, H, H, B * n1, n0 * H, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_swap(p, w, o, n1, n0, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
    }
    return FFT3D_OK;
}

int fft3d_c2r(fft3d_handle p, void* in, float* out, void* stream)
{
    if (!p || !in || !out || p->dtype == FFT3D_F64) return fail(FFT3D_ERR_INVALID_ARG);
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return fail(FFT3D_ERR_MISALIGNED);
    const size_t in_bytes = (size_t)p->batch * p->M * sizeof(float2);
    const size_t out_bytes = real_bytes(p);
    const bool preserve = p->flags & FFT3D_FLAG_PRESERVE_INPUT;
    const bool in_place = (p->flags & FFT3D_FLAG_PADDED_REAL) && in == (void*)out && !preserve;
    if (!in_place && overlaps(in, in_bytes, out, out_bytes)) return fail(FFT3D_ERR_INVALID_ARG);
    const bool xpose = p->flags & FFT3D_FLAG_EXPLICIT_TRANSPOSE;
    if ((xpose || preserve) && !p->workspace) return fail(FFT3D_ERR_NO_WORKSPACE);
    cudaStream_t s = (cudaStream_t)stream;
    const long long H = p->H, n0 = p->n0, n1 = p->n1, B = p->batch;
    float2* x = (float2*)in;
    if (preserve && p->workspace && overlaps(in, in_bytes, p->workspace, in_bytes)) return fail(FFT3D_ERR_INVALID_ARG);
    if (preserve) {
        // the first column pass reads the input and writes the workspace; the
        // rest runs there (the row c2r only reads its input)
        float2* w = (float2*)p->workspace;
        float2* src = x;
        if (n0 > 1) {
            if (run_col(p, p->ax0, +1, src, p->P, p->P, B, p->M, s, w) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
            src = w;
        }
        if (p->cplane) {
            if (run_cplane(p, +1, src, out, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
            return FFT3D_OK;
        }
        if (n1 > 1) {
            if (run_col(p, p->ax1, +1, src, H, H, B * n0, n1 * H, s, src == w ? nullptr : w) != cudaSuccess)
                return fail(FFT3D_ERR_CUDA);
            src = w;
        }
        if (run_row(p, +1, src, out, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        return FFT3D_OK;
    }
    if (!xpose && p->cplane) {
        if (run_col(p, p->ax0, +1, x, p->P, p->P, B, p->M, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_cplane(p, +1, x, out, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        return FFT3D_OK;
    }
    if (!xpose && p->plane) {
        if (run_col(p, p->ax0, +1, x, p->P, p->P, B, p->M, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_plane(p, +1, x, out, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        return FFT3D_OK;
    }
    if (!xpose) {
        if (run_col(p, p->ax0, +1, x, p->P, p->P, B, p->M, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_col(p, p->ax1, +1, x, H, H, B * n0, n1 * H, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_row(p, +1, x, out, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        return FFT3D_OK;
    }
    float2* w = (float2*)p->workspace;
    if (!(p->flags & FFT3D_FLAG_TRANSPOSE_BACK)) {
        // input is (n1, n0, H): n0 pass on the middle axis, transpose back to (n0, n1, H)
        if (run_col(p, p->ax0, +1, x, H, H, B * n1, n0 * H, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_swap(p, x, w, n1, n0, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_col(p, p->ax1, +1, w, H, H, B * n0, n1 * H, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_row(p, +1, w, out, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
    } else {
        if (run_swap(p, x, w, n0, n1, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_col(p, p->ax0, +1, w, H, H, B * n1, n0 * H, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_swap(p, w, x, n1, n0, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_col(p, p->ax1, +1, x, H, H, B * n0, n1 * H, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        if (run_row(p, +1, x, out, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
    }
    return FFT3D_OK;
}

// FFT3D_F64 plans: the transpose-free pass sequence of fft3d_r2c / fft3d_c2r
// (rows, n1 columns at stride H, n0 columns at stride n1 H; the inverse in
// reverse order), every pass on the FP64 runtime-length kernels.
int fft3d_r2c_f64(fft3d_handle p, const double* in, void* out, void* stream)
{
    if (!p || !in || !out || p->dtype != FFT3D_F64) return fail(FFT3D_ERR_INVALID_ARG);
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return fail(FFT3D_ERR_MISALIGNED);
    const size_t in_bytes = (size_t)p->batch * p->n0 * p->n1 * p->n2 * sizeof(double);
    const size_t out_bytes = (size_t)p->batch * p->M * sizeof(double2);
    if (overlaps(in, in_bytes, out, out_bytes)) return fail(FFT3D_ERR_INVALID_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    const long long H = p->H, n0 = p->n0, n1 = p->n1, B = p->batch;
    double2* o = (double2*)out;
    const bool odd = p->n2 & 1;
    RowArgs64 ra{in, out, B * n0 * n1, p->ax2.d_tw64, p->d_twpack64, odd ? (long long)p->n2 : (long long)p->n2 / 2};
    if ((odd ? generic_row_odd64(ra, p->ax2.gen64, -1, s) : generic_row64(ra, p->ax2.gen64, -1, s)) != cudaSuccess)
        return fail(FFT3D_ERR_CUDA);
    if (n1 > 1) {
        ColArgs64 ca{o, H, H, B * n0, n1 * H, p->ax1.d_tw64, nullptr};
        if (generic_col64(ca, p->ax1.gen64, -1, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
    }
    if (n0 > 1) {
        ColArgs64 ca{o, p->P, p->P, B, p->M, p->ax0.d_tw64, nullptr};
        if (generic_col64(ca, p->ax0.gen64, -1, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
    }
    return FFT3D_OK;
}

int fft3d_c2r_f64(fft3d_handle p, void* in, double* out, void* stream)
{
    if (!p || !in || !out || p->dtype != FFT3D_F64) return fail(FFT3D_ERR_INVALID_ARG);
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return fail(FFT3D_ERR_MISALIGNED);
    const size_t in_bytes = (size_t)p->batch * p->M * sizeof(double2);
    const size_t out_bytes = (size_t)p->batch * p->n0 * p->n1 * p->n2 * sizeof(double);
    if (overlaps(in, in_bytes, out, out_bytes)) return fail(FFT3D_ERR_INVALID_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    const long long H = p->H, n0 = p->n0, n1 = p->n1, B = p->batch;
    double2* x = (double2*)in;
    if (n0 > 1) {
        ColArgs64 ca{x, p->P, p->P, B, p->M, p->ax0.d_tw64, nullptr};
        if (generic_col64(ca, p->ax0.gen64, +1, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
    }
    if (n1 > 1) {
        ColArgs64 ca{x, H, H, B * n0, n1 * H, p->ax1.d_tw64, nullptr};
        if (generic_col64(ca, p->ax1.gen64, +1, s) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
    }
    const bool odd = p->n2 & 1;
    RowArgs64 ra{in, out, B * n0 * n1, p->ax2.d_tw64, p->d_twpack64, odd ? (long long)p->n2 : (long long)p->n2 / 2};
    if ((odd ? generic_row_odd64(ra, p->ax2.gen64, +1, s) : generic_row64(ra, p->ax2.gen64, +1, s)) != cudaSuccess)
        return fail(FFT3D_ERR_CUDA);
    return FFT3D_OK;
}

int fft3d_energy(fft3d_handle p, const void* spec, double* total, double* shells, int nbins, void* stream)
{
    if (!p || !spec || nbins < 1 || nbins > 8192 || (!total && !shells) || p->dtype == FFT3D_F64)
        return fail(FFT3D_ERR_INVALID_ARG);
    if (((uintptr_t)spec & 15) || ((uintptr_t)total & 7) || ((uintptr_t)shells & 7)) return fail(FFT3D_ERR_MISALIGNED);
    const size_t need = energy_scratch_doubles(p->batch, (long long)p->n0 * p->n1, nbins);
    if (need > p->energy_doubles) {
        cudaDeviceSynchronize();
        cudaFree(p->d_energy);
        p->d_energy = nullptr;
        p->energy_doubles = 0;
        if (cudaMalloc((void**)&p->d_energy, need * sizeof(double)) != cudaSuccess) return fail(FFT3D_ERR_ALLOC);
        p->energy_doubles = need;
    }
    if (launch_energy(spec, p->n0, p->n1, p->n2, p->batch, nbins, p->d_energy, total, shells,
                      (cudaStream_t)stream) != cudaSuccess)
        return fail(FFT3D_ERR_CUDA);
    return FFT3D_OK;
}

// ---------------------------------------------------------------------------
// Pseudo-spectral nonlinear term.
// ---------------------------------------------------------------------------
struct fft3d_nl_s {
    fft3d_plan_s* plan = nullptr;  // batch-1 plan: twiddles and kernel choices
    void* workspace = nullptr;     // 3 * M complex, lent by the caller
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void* g_uhat = nullptr;  // operands the graph was captured with
    void* g_nhat = nullptr;
    void* g_ws = nullptr;
    // plane chunking of the middle passes (n1 inverse, rows, n1 forward): the
    // planes j0 in chunks of `chunk`, each chunk's three passes back to back
    // so their operands stay in L2; with streams = 2 alternate chunks run on a
    // second stream (captured graphs only) so one chunk's passes fill the
    // other's ramp-up and tail
    int chunk = 0;  // planes per chunk (0: all n0 planes in one chunk)
    int streams = 1;
    cudaStream_t s2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace {

// s2: the second stream of the two-stream chunk order, or nullptr (one stream)
cudaError_t enqueue_nonlinear(fft3d_nl_s* nl, const void* uhat, void* nhat, cudaStream_t s, cudaStream_t s2)
{
    fft3d_plan_s* p = nl->plan;
    const long long H = p->H, n0 = p->n0, n1 = p->n1, M = p->M, P = p->P;
    float2* W = (float2*)nl->workspace;
    float2* U = (float2*)const_cast<void*>(uhat);
    float2* Nh = (float2*)nhat;
    cudaError_t e;
    // 1. n0 inverse of the three fields, out of place into the workspace (uhat is preserved)
    if (p->n0 > 1) {
        ColArgs c{U, P, P, 3, M, p->ax0.d_tw, 1.0f, p->d_status, W, 0};
        if ((e = launch_col_args(p, p->ax0, +1, c, s)) != cudaSuccess) return e;
    } else if ((e = cudaMemcpyAsync(W, U, 3 * M * sizeof(float2), cudaMemcpyDeviceToDevice, s)) != cudaSuccess) {
        return e;
    }
    // The forward passes visit only what the 2/3 rule keeps; everything else
    // is zero already.  The rows write zeros at k2 >= keep2, so the n1 pass
    // transforms the columns k2 < keep2 alone (a column of zeros stays zero)
    // and zeroes the k1 the rule drops; the n0 pass then transforms only the
    // columns whose k1 and k2 are both kept (two blocks of k1: 0 .. A-1 and
    // n1-B .. n1-1), the others being zero in place.
    const long long keep2 = (p->n2 + 2) / 3;
    // 2-4, per chunk of planes j0 (all fields of a plane together):
    //   n1 inverse of the three fields, in place;
    //   rows: three c2r, six products, six r2c with the 2/3 rule on k2;
    //   n1 forward of the six products over k2 < keep2, 2/3 rule on k1.
    const long long chunk = nl->chunk > 0 && nl->chunk < n0 ? nl->chunk : n0;
    const bool two = s2 != nullptr && chunk < n0;
    if (two) {
        if ((e = cudaEventRecord(nl->ev_fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s2, nl->ev_fork, 0)) != cudaSuccess) return e;
    }
    for (long long j0 = 0, g = 0; j0 < n0; j0 += chunk, ++g) {
        const long long cc = n0 - j0 < chunk ? n0 - j0 : chunk;
        const long long off = j0 * n1 * H;
        cudaStream_t sc = (two && (g & 1)) ? s2 : s;
        // all planes in one chunk: the fields' planes are one evenly strided
        // batch (field stride M = n0 planes), which every column form takes
        const bool whole = cc == n0;
        if (p->n1 > 1) {
            ColArgs c{W + off, H, H, whole ? 3 * n0 : cc, n1 * H, p->ax1.d_tw, 1.0f, p->d_status, nullptr, 0};
            c.nb2 = whole ? 1 : 3;
            c.Bs2 = whole ? 0 : M;
            if ((e = launch_col_args(p, p->ax1, +1, c, sc)) != cudaSuccess) return e;
        }
        NlRowArgs r{W + off, Nh + off, cc * n1, M, p->ax2.d_tw, p->d_twpack, (int)keep2};
        if ((e = p->ax2.spec->nl(r, sc)) != cudaSuccess) return e;
        if (p->n1 > 1) {
            ColArgs c{Nh + off, H, keep2, whole ? 6 * n0 : cc, n1 * H, p->ax1.d_tw, 1.0f, p->d_status, nullptr, 1};
            c.nb2 = whole ? 1 : 6;
            c.Bs2 = whole ? 0 : M;
            if ((e = launch_col_args(p, p->ax1, -1, c, sc)) != cudaSuccess) return e;
        }
    }
    if (two) {
        if ((e = cudaEventRecord(nl->ev_join, s2)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, nl->ev_join, 0)) != cudaSuccess) return e;
    }
    // 5. n0 forward of the kept (k1, k2) columns, 2/3 rule on k0 and the 1/N normalisation
    const long long A = (n1 + 2) / 3, B = (n1 - 1) / 3;  // kept k1 >= 0 (3 k1 < n1), kept k1 < 0 (3 |k1| < n1)
    const long long starts[2] = {0, n1 - B}, counts[2] = {A, B};
    for (int q = 0; q < 2; ++q) {
        if (counts[q] <= 0 || (q == 1 && n1 == 1)) continue;
        ColArgs c{Nh + starts[q] * H, P, keep2, counts[q], H, p->ax0.d_tw, 1.0f / (float)p->N, p->d_status, nullptr, 1};
        c.nb2 = 6;
        c.Bs2 = M;
        if ((e = launch_col_args(p, p->ax0, -1, c, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The second stream of the two-stream chunk order (created on first use, on
// the plan's device), or nullptr when the plan runs on one stream.
cudaStream_t nl_second_stream(fft3d_nl_s* nl)
{
    if (nl->streams < 2) return nullptr;
    if (!nl->s2) {
        int cur = 0;
        if (cudaGetDevice(&cur) != cudaSuccess) return nullptr;
        if (cur != nl->plan->device && cudaSetDevice(nl->plan->device) != cudaSuccess) return nullptr;
        cudaStream_t st = nullptr;
        cudaEvent_t a = nullptr, b = nullptr;
        const bool ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
                        cudaEventCreateWithFlags(&a, cudaEventDisableTiming) == cudaSuccess &&
                        cudaEventCreateWithFlags(&b, cudaEventDisableTiming) == cudaSuccess;
        if (cur != nl->plan->device) cudaSetDevice(cur);
        if (!ok) {
            if (st) cudaStreamDestroy(st);
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
            return nullptr;
        }
        nl->s2 = st;
        nl->ev_fork = a;
        nl->ev_join = b;
    }
    return nl->s2;
}

// Kernel nodes of a captured graph, or -1.
int graph_kernel_nodes(cudaGraph_t g)
{
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return -1;
    std::vector<cudaGraphNode_t> nodes(n);
    if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return -1;
    int k = 0;
    for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess) return -1;
        k += t == cudaGraphNodeTypeKernel;
    }
    return k;
}

// Launches enqueue_nonlinear issues with this plan's kernel forms: the n0
// inverse pass; per chunk of planes the n1 inverse pass, the fused rows and
// the n1 forward pass; the n0 forward pass over the two kept k1 blocks.  A
// pass over an outer batch of fields is one launch where the axis' column
// path takes the batch, else one per field.
int nonlinear_launch_count(const fft3d_nl_s* nl)
{
    const fft3d_plan_s* p = nl->plan;
    const long long n0 = p->n0, n1 = p->n1, A = (n1 + 2) / 3, B = (n1 - 1) / 3;
    auto outer = [p](const Axis& a) { return !(uses_generic(p, a, false) || a.tc || !a.spec); };
    const long long chunk = nl->chunk > 0 && nl->chunk < n0 ? nl->chunk : n0;
    const long long chunks = (n0 + chunk - 1) / chunk;
    const bool o1 = chunks == 1 || outer(p->ax1);
    const long long mid = (n1 > 1) * (o1 ? 2 : 9) + 1;
    const int blocks = (A > 0) + (B > 0 && n1 > 1);
    return (int)((n0 > 1) + chunks * mid + blocks * (outer(p->ax0) ? 1 : 6));
}

void drop_graph(fft3d_nl_s* nl)
{
    if (nl->exec) cudaGraphExecDestroy(nl->exec);
    if (nl->graph) cudaGraphDestroy(nl->graph);
    nl->exec = nullptr;
    nl->graph = nullptr;
    nl->g_uhat = nullptr;
    nl->g_nhat = nullptr;
    nl->g_ws = nullptr;
}

}  // namespace

fft3d_nl_handle fft3d_nonlinear_plan(int n0, int n1, int n2)
{
    fft3d_handle p = fft3d_plan_variant(n0, n1, n2, FFT3D_F32, 1, 0);
    if (!p) return nullptr;
    // the 1D passes are per axis; the 2/3 rule needs n1 and n0 passes that apply it
    if (!p->ax2.spec || p->ax2.spec->nl == nullptr || (p->flags & FFT3D_FLAG_GENERIC)) {
        fft3d_destroy(p);
        fail(FFT3D_ERR_UNSUPPORTED_SIZE);
        return nullptr;
    }
    fft3d_nl_s* nl = new (std::nothrow) fft3d_nl_s();
    if (!nl) {
        fft3d_destroy(p);
        fail(FFT3D_ERR_ALLOC);
        return nullptr;
    }
    nl->plan = p;
    return nl;
}

size_t fft3d_nonlinear_workspace_bytes(fft3d_nl_handle nl)
{
    return nl ? (size_t)3 * (size_t)nl->plan->M * sizeof(float2) : 0;
}

int fft3d_nonlinear_set_workspace(fft3d_nl_handle nl, void* dev_ptr)
{
    if (!nl) return fail(FFT3D_ERR_INVALID_ARG);
    if (dev_ptr && ((uintptr_t)dev_ptr & 255)) return fail(FFT3D_ERR_MISALIGNED);
    nl->workspace = dev_ptr;
    return FFT3D_OK;
}

int fft3d_nonlinear_exec(fft3d_nl_handle nl, const void* uhat, void* nhat, void* stream)
{
    if (!nl || !uhat || !nhat) return fail(FFT3D_ERR_INVALID_ARG);
    if (!nl->workspace) return fail(FFT3D_ERR_NO_WORKSPACE);
    if (((uintptr_t)uhat & 15) || ((uintptr_t)nhat & 15)) return fail(FFT3D_ERR_MISALIGNED);
    const size_t M8 = (size_t)nl->plan->M * sizeof(float2);
    if (overlaps(uhat, 3 * M8, nhat, 6 * M8) || overlaps(uhat, 3 * M8, nl->workspace, 3 * M8) ||
        overlaps(nhat, 6 * M8, nl->workspace, 3 * M8))
        return fail(FFT3D_ERR_INVALID_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    if (!s) {  // the legacy default stream cannot be captured: launch directly, on one stream
        return enqueue_nonlinear(nl, uhat, nhat, s, nullptr) == cudaSuccess ? FFT3D_OK : fail(FFT3D_ERR_CUDA);
    }
    if (!(nl->exec && nl->g_uhat == uhat && nl->g_nhat == nhat && nl->g_ws == nl->workspace)) {
        drop_graph(nl);
        cudaStream_t s2 = nl_second_stream(nl);
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        const cudaError_t e = enqueue_nonlinear(nl, uhat, nhat, s, s2);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(s, &g);
        if (e != cudaSuccess || e2 != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            return fail(FFT3D_ERR_CUDA);
        }
        nl->graph = g;
        if (cudaGraphInstantiate(&nl->exec, g, 0) != cudaSuccess) {
            drop_graph(nl);
            return fail(FFT3D_ERR_CUDA);
        }
        nl->g_uhat = uhat;
        nl->g_nhat = nhat;
        nl->g_ws = nl->workspace;
    }
    return cudaGraphLaunch(nl->exec, s) == cudaSuccess ? FFT3D_OK : fail(FFT3D_ERR_CUDA);
}

// ---------------------------------------------------------------------------
// Pseudo-spectral Navier-Stokes step (Heun) around the nonlinear term.
// ---------------------------------------------------------------------------
struct fft3d_ns_s {
    fft3d_nl_s* nl = nullptr;      // the nonlinear term (and its batch-1 plan)
    void* workspace = nullptr;     // [u* 3M][acc 3M][nhat 6M][nonlinear scratch 3M]
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void* g_u = nullptr;     // operands the graph was captured with
    void* g_ws = nullptr;
    float g_nu = 0.f, g_dt = 0.f;
};

namespace {

void drop_ns_graph(fft3d_ns_s* ns)
{
    if (ns->exec) cudaGraphExecDestroy(ns->exec);
    if (ns->graph) cudaGraphDestroy(ns->graph);
    ns->exec = nullptr;
    ns->graph = nullptr;
    ns->g_u = nullptr;
    ns->g_ws = nullptr;
}

// s2: as for enqueue_nonlinear
cudaError_t enqueue_ns_step(fft3d_ns_s* ns, float2* u, float nu, float dt, cudaStream_t s, cudaStream_t s2)
{
    const fft3d_plan_s* p = ns->nl->plan;
    const long long M = p->M;
    float2* w = (float2*)ns->workspace;
    NsArgs a{u, w, w + 3 * M, w + 6 * M, p->n0, p->n1, p->n2, (int)p->H, M, nu, dt};
    cudaError_t e;
    if ((e = enqueue_nonlinear(ns->nl, u, w + 6 * M, s, s2)) != cudaSuccess) return e;
    if ((e = launch_ns_stage(a, 1, s)) != cudaSuccess) return e;
    if ((e = enqueue_nonlinear(ns->nl, w, w + 6 * M, s, s2)) != cudaSuccess) return e;
    return launch_ns_stage(a, 2, s);
}

}  // namespace

fft3d_ns_handle fft3d_ns_plan(int n0, int n1, int n2)
{
    fft3d_nl_handle nl = fft3d_nonlinear_plan(n0, n1, n2);
    if (!nl) return nullptr;
    fft3d_ns_s* ns = new (std::nothrow) fft3d_ns_s();
    if (!ns) {
        fft3d_nonlinear_destroy(nl);
        fail(FFT3D_ERR_ALLOC);
        return nullptr;
    }
    ns->nl = nl;
    return ns;
}

size_t fft3d_ns_workspace_bytes(fft3d_ns_handle ns)
{
    return ns ? (size_t)15 * (size_t)ns->nl->plan->M * sizeof(float2) : 0;
}

int fft3d_ns_set_workspace(fft3d_ns_handle ns, void* dev_ptr)
{
    if (!ns) return fail(FFT3D_ERR_INVALID_ARG);
    if (dev_ptr && ((uintptr_t)dev_ptr & 255)) return fail(FFT3D_ERR_MISALIGNED);
    ns->workspace = dev_ptr;
    ns->nl->workspace = dev_ptr ? (char*)dev_ptr + (size_t)12 * ns->nl->plan->M * sizeof(float2) : nullptr;
    return FFT3D_OK;
}

int fft3d_ns_step(fft3d_ns_handle ns, void* uhat, float nu, float dt, void* stream)
{
    if (!ns || !uhat || !(nu >= 0.f) || !(dt > 0.f)) return fail(FFT3D_ERR_INVALID_ARG);
    if (!ns->workspace) return fail(FFT3D_ERR_NO_WORKSPACE);
    if ((uintptr_t)uhat & 15) return fail(FFT3D_ERR_MISALIGNED);
    const size_t M8 = (size_t)ns->nl->plan->M * sizeof(float2);
    if (overlaps(uhat, 3 * M8, ns->workspace, 15 * M8)) return fail(FFT3D_ERR_INVALID_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    float2* u = (float2*)uhat;
    if (!s) return enqueue_ns_step(ns, u, nu, dt, s, nullptr) == cudaSuccess ? FFT3D_OK : fail(FFT3D_ERR_CUDA);
    if (!(ns->exec && ns->g_u == uhat && ns->g_ws == ns->workspace && ns->g_nu == nu && ns->g_dt == dt)) {
        drop_ns_graph(ns);
        cudaStream_t s2 = nl_second_stream(ns->nl);
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        const cudaError_t e = enqueue_ns_step(ns, u, nu, dt, s, s2);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(s, &g);
        if (e != cudaSuccess || e2 != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            return fail(FFT3D_ERR_CUDA);
        }
        ns->graph = g;
        if (cudaGraphInstantiate(&ns->exec, g, 0) != cudaSuccess) {
            drop_ns_graph(ns);
            return fail(FFT3D_ERR_CUDA);
        }
        ns->g_u = uhat;
        ns->g_ws = ns->workspace;
        ns->g_nu = nu;
        ns->g_dt = dt;
    }
    return cudaGraphLaunch(ns->exec, s) == cudaSuccess ? FFT3D_OK : fail(FFT3D_ERR_CUDA);
}

int fft3d_ns_set_chunking(fft3d_ns_handle ns, int planes, int streams)
{
    if (!ns) return fail(FFT3D_ERR_INVALID_ARG);
    const int r = fft3d_nonlinear_set_chunking(ns->nl, planes, streams);
    if (r == FFT3D_OK) drop_ns_graph(ns);
    return r;
}

int fft3d_ns_launches(fft3d_ns_handle ns)
{
    if (!ns) return fail(FFT3D_ERR_INVALID_ARG);
    if (ns->graph) {
        const int k = graph_kernel_nodes(ns->graph);
        if (k >= 0) return k;
    }
    return 2 * nonlinear_launch_count(ns->nl) + 2;
}

void fft3d_ns_destroy(fft3d_ns_handle ns)
{
    if (!ns) return;
    cudaDeviceSynchronize();
    drop_ns_graph(ns);
    fft3d_nonlinear_destroy(ns->nl);
    delete ns;
}

int fft3d_nonlinear_launches(fft3d_nl_handle nl)
{
    if (!nl) return fail(FFT3D_ERR_INVALID_ARG);
    if (nl->graph) {
        const int k = graph_kernel_nodes(nl->graph);
        if (k >= 0) return k;
    }
    return nonlinear_launch_count(nl);
}

int fft3d_nonlinear_set_chunking(fft3d_nl_handle nl, int planes, int streams)
{
    if (!nl || planes < 0 || streams < 1 || streams > 2) return fail(FFT3D_ERR_INVALID_ARG);
    nl->chunk = planes;
    nl->streams = streams;
    drop_graph(nl);  // the next call captures the new order
    return FFT3D_OK;
}

int fft3d_nonlinear_get_chunking(fft3d_nl_handle nl, int* planes, int* streams)
{
    if (!nl || !planes || !streams) return fail(FFT3D_ERR_INVALID_ARG);
    *planes = nl->chunk;
    *streams = nl->streams;
    return FFT3D_OK;
}

void fft3d_nonlinear_destroy(fft3d_nl_handle nl)
{
    if (!nl) return;
    cudaDeviceSynchronize();
    drop_graph(nl);
    if (nl->s2) cudaStreamDestroy(nl->s2);
    if (nl->ev_fork) cudaEventDestroy(nl->ev_fork);
    if (nl->ev_join) cudaEventDestroy(nl->ev_join);
    fft3d_destroy(nl->plan);
    delete nl;
}

// ---------------------------------------------------------------------------
// Autotuner and shape choices.
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

template <class F>
float time_pass(F&& f, int reps, cudaStream_t s)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    f();  // warm-up (also first-use set-up of the kernel)
    cudaEventRecord(a, s);
    for (int i = 0; i < reps; ++i) f();
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return (cudaGetLastError() == cudaSuccess) ? ms / reps : 1e30f;
}

}  // namespace

extern "C" {

int fft3d_get_choices(fft3d_handle p, int* c)
{
    if (!p || !c) return fail(FFT3D_ERR_INVALID_ARG);
    c[0] = p->choice_w0;
    c[1] = p->choice_w1;
    c[2] = p->choice_rows;
    c[3] = p->choice_tma;
    c[4] = p->choice_tma1;
    return FFT3D_OK;
}

int fft3d_set_choices(fft3d_handle p, const int* c)
{
    // column forms: 0 plain, 1 TMA ring, 2 + i the axis's i-th cluster-split kernel (must exist),
    // 4 TMA-fed cluster split, 5 residue split, 6 TMA row pairs with two columns per thread
    auto form_ok = [](int f, const Axis& a) {
        return f == 0 || f == 1 || ((f == 2 || f == 3) && a.split[f - 2]) || (f == 4 && a.tsplit) ||
               (f == 5 && a.l2split) || (f == 6 && a.spec && a.spec->tma_pair2_fwd);
    };
    if (!p || !c || c[0] < 0 || c[1] < 0 || c[2] < 0 || !form_ok(c[3], p->ax0) || !form_ok(c[4], p->ax1))
        return fail(FFT3D_ERR_INVALID_ARG);
    p->choice_w0 = c[0];
    p->choice_w1 = c[1];
    p->choice_rows = c[2];
    p->choice_tma = c[3];
    p->choice_tma1 = c[4];
    return FFT3D_OK;
}

int fft3d_get_plane_choice(fft3d_handle p)
{
    if (!p) return -fail(FFT3D_ERR_INVALID_ARG);
    return p->cplane ? p->cplane->C : 0;
}

int fft3d_set_plane_choice(fft3d_handle p, int cluster)
{
    if (!p || cluster < 0) return fail(FFT3D_ERR_INVALID_ARG);
    if (cluster == 0) {
        p->cplane = nullptr;
        return FFT3D_OK;
    }
    if (!cplane_allowed(p)) return fail(FFT3D_ERR_INVALID_ARG);
    const CPlaneEntry* e = cplane_for(p->n2 / 2, p->n1, cluster);
    if (!e) return fail(FFT3D_ERR_UNSUPPORTED_SIZE);
    p->cplane = e;
    return FFT3D_OK;
}

int fft3d_autotune(fft3d_handle p, float* real, void* cplx, int reps, void* stream)
{
    if (!p || !real || !cplx || p->dtype == FFT3D_F64) return fail(FFT3D_ERR_INVALID_ARG);
    if (((uintptr_t)real & 15) || ((uintptr_t)cplx & 15)) return fail(FFT3D_ERR_MISALIGNED);
    if (p->flags & (FFT3D_FLAG_GENERIC | FFT3D_FLAG_EXPLICIT_TRANSPOSE)) return FFT3D_OK;  // nothing to choose
    if (reps < 1) reps = 5;
    cudaStream_t s = (cudaStream_t)stream;
    const bool prof = p->profiling;
    p->profiling = false;
    const long long H = p->H, n0 = p->n0, n1 = p->n1, B = p->batch;
    float2* X = (float2*)cplx;
    // rows per CTA of the row kernels
    if (p->ax2.spec && p->ax2.spec->row_warp) {
        const int R = p->ax2.spec->row_rows, T = p->ax2.L / p->ax2.spec->row_E;
        float best = 1e30f;
        int pick = 0;
        for (int r = R; r >= 1; r /= 2) {
            if ((T * r) % 32) break;
            p->choice_rows = r;
            const float t = time_pass([&] { run_row(p, -1, real, X, s); }, reps, s);
            if (t < best) best = t, pick = r;
        }
        p->choice_rows = pick;
    }
    // n1 pass: the TMA kernel (rows or row pairs) or the plain kernel at several widths
    if (p->ax1.L > 1 && p->ax1.spec && !p->ax1.tc) {
        float best = 1e30f;
        int pick = 0, pick_tma = 0;
        if (tma_ok(p, p->ax1, H, H, n1 * H)) {
            p->choice_tma1 = 1;
            best = time_pass([&] { run_col(p, p->ax1, -1, X, H, H, B * n0, n1 * H, s); }, reps, s);
            pick_tma = 1;
        }
        p->choice_tma1 = 0;
        for (int w = p->ax1.spec->col_W; w >= 4 && w * 4 >= p->ax1.spec->col_W; w /= 2) {
            p->choice_w1 = w;
            const float t = time_pass([&] { run_col(p, p->ax1, -1, X, H, H, B * n0, n1 * H, s); }, reps, s);
            if (t < best) best = t, pick = w, pick_tma = 0;
        }
        p->choice_w1 = pick;
        for (int f = 2; f <= 6; ++f) {  // split kernels: cluster (plain, TMA-fed), residues through L2; 2-column row pairs
            if (f < 4 ? !p->ax1.split[f - 2]
                      : f == 4 ? (!p->ax1.tsplit || H % 2 || H < 16)
                               : f == 5 ? !p->ax1.l2split
                                        : (!p->ax1.spec->tma_pair2_fwd || tma_mode(p, p->ax1, H, H, n1 * H) != 2))
                continue;
            p->choice_tma1 = f;
            const float t = time_pass([&] { run_col(p, p->ax1, -1, X, H, H, B * n0, n1 * H, s); }, reps, s);
            if (t < best) best = t, pick_tma = f;
        }
        p->choice_tma1 = pick_tma;
    }
    // n0 pass: the TMA kernel or the plain kernel at several widths
    if (p->ax0.L > 1 && p->ax0.spec && !p->ax0.tc) {
        float best = 1e30f;
        int pick_w = 0, pick_tma = 0;
        if (tma_ok(p, p->ax0, p->P, p->P, p->M)) {
            p->choice_tma = 1;
            best = time_pass([&] { run_col(p, p->ax0, -1, X, p->P, p->P, B, p->M, s); }, reps, s);
            pick_tma = 1;
        }
        p->choice_tma = 0;
        for (int w = p->ax0.spec->col_W; w >= 4 && w * 4 >= p->ax0.spec->col_W; w /= 2) {
            p->choice_w0 = w;
            const float t = time_pass([&] { run_col(p, p->ax0, -1, X, p->P, p->P, B, p->M, s); }, reps, s);
            if (t < best) best = t, pick_w = w, pick_tma = 0;
        }
        p->choice_w0 = pick_w;
        for (int f = 2; f <= 5; ++f) {  // split kernels: cluster (plain, TMA-fed), residues through L2
            if (f < 4 ? !p->ax0.split[f - 2]
                      : f == 4 ? (!p->ax0.tsplit || p->P % 2 || p->P < 16) : !p->ax0.l2split)
                continue;
            p->choice_tma = f;
            const float t = time_pass([&] { run_col(p, p->ax0, -1, X, p->P, p->P, B, p->M, s); }, reps, s);
            if (t < best) best = t, pick_tma = f;
        }
        p->choice_tma = pick_tma;
    }
    // plane form: separate row and n1 passes, or a cluster plane kernel of
    // each instantiated cluster size, timed over a whole r2c + c2r
    if (cplane_allowed(p) && cplane_for(p->n2 / 2, p->n1, 0)) {
        int nc = 0;
        const CPlaneEntry* ce = cplane_entries(&nc);
        const CPlaneEntry* best_e = nullptr;
        p->cplane = nullptr;
        float best = time_pass([&] { fft3d_r2c(p, real, cplx, stream); fft3d_c2r(p, cplx, real, stream); }, reps, s);
        for (int i = 0; i < nc; ++i) {
            if (ce[i].LR != p->n2 / 2 || ce[i].LC != p->n1) continue;
            p->cplane = &ce[i];
            const float t = time_pass([&] { fft3d_r2c(p, real, cplx, stream); fft3d_c2r(p, cplx, real, stream); }, reps, s);
            if (t < best) best = t, best_e = &ce[i];
        }
        p->cplane = best_e;
    }
    p->profiling = prof;
    p->desc = describe_plan(p);
    if (log_enabled())
        std::fprintf(stderr, "fft3d: autotune %dx%dx%d: choices {%d, %d, %d, %d, %d} plane C=%d: %s\n", p->n0, p->n1,
                     p->n2, p->choice_w0, p->choice_w1, p->choice_rows, p->choice_tma, p->choice_tma1,
                     p->cplane ? p->cplane->C : 0, p->desc.c_str());
    return cudaGetLastError() == cudaSuccess ? FFT3D_OK : fail(FFT3D_ERR_CUDA);
}

// ---------------------------------------------------------------------------
// Grouped transforms of uneven sizes: one plan per size (its fields form the
// plan's batch), each size on its own stream, forked from and joined back
// into the caller's stream; on a non-default stream the whole group is
// captured once per operand set into a CUDA graph and replayed.
// ---------------------------------------------------------------------------
struct fft3d_group_s {
    std::vector<fft3d_plan_s*> plans;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    struct Graph {
        std::vector<const void*> in;
        std::vector<void*> mid;
        std::vector<void*> out;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
    } graphs[3];  // forward, inverse, forward + inverse
    // work-table form: every size has compiled item bodies
    bool wt_ok = false;
    int form = 0;                  // FFT3D_GROUP_STREAMS, FFT3D_GROUP_WORK_TABLE (or the test form)
    WtCounters* d_ctr = nullptr;   // counters of one launch (zeroed before it)
};

namespace {

void group_free(fft3d_group_s* g)
{
    cudaFree(g->d_ctr);
    for (auto& gr : g->graphs) {
        if (gr.exec) cudaGraphExecDestroy(gr.exec);
        if (gr.graph) cudaGraphDestroy(gr.graph);
    }
    for (auto* p : g->plans) fft3d_destroy(p);
    for (auto st : g->streams) cudaStreamDestroy(st);
    for (auto e : g->joins) cudaEventDestroy(e);
    if (g->fork) cudaEventDestroy(g->fork);
    delete g;
}

// Segments of one pass of every size (largest first) into the work table.
// pass: 0 rows, 1 n1, 2 n0; prev[i]: the segment size i's pass depends on
// (-1: none); on return prev[i] is this pass's segment of size i.
int wt_add_pass(const fft3d_group_s* g, WtTable& t, int pass, int dir, const void* const* rin, void* const* rout,
                void* const* spec, std::vector<int>& prev)
{
    std::vector<size_t> order(g->plans.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        return g->plans[a]->batch * g->plans[a]->N > g->plans[b]->batch * g->plans[b]->N;
    });
    for (size_t i : order) {
        const fft3d_plan_s* p = g->plans[i];
        if (t.nseg >= kWtMaxSeg) return FFT3D_ERR_UNSUPPORTED_SIZE;
        WtSeg& sg = t.seg[t.nseg];
        sg = WtSeg{};
        int per = 0;
        const long long B = p->batch, n0 = p->n0, n1 = p->n1, H = p->H;
        if (pass == 0) {
            sg.body = wt_body_index(true, p->n2 / 2, dir, &per);
            sg.rows = B * n0 * n1;
            sg.items = (sg.rows + per - 1) / per;
            sg.in = dir < 0 ? rin[i] : spec[i];
            sg.out = dir < 0 ? spec[i] : rout[i];
            sg.rs = p->n2 / 2;
            sg.tw = p->ax2.d_tw;
            sg.twpack = p->d_twpack;
        } else {
            const Axis& a = pass == 1 ? p->ax1 : p->ax0;
            sg.body = wt_body_index(false, a.L, dir, &per);
            sg.data = (float2*)spec[i];
            sg.S = pass == 1 ? H : p->P;
            sg.C = sg.S;
            sg.nb = pass == 1 ? B * n0 : B;
            sg.Bs = pass == 1 ? n1 * H : p->M;
            sg.items = sg.nb * ((sg.C + per - 1) / per);
            sg.tw = a.d_tw;
        }
        if (sg.body < 0) return FFT3D_ERR_UNSUPPORTED_SIZE;
        sg.dep = prev[i];
        sg.need = sg.dep >= 0 ? t.seg[sg.dep].items : 0;
        sg.first = t.total;
        t.total += sg.items;
        prev[i] = t.nseg++;
    }
    return FFT3D_OK;
}

// The work table of a forward (dir < 0: in = real, mid = spectra), an inverse
// (dir > 0: mid = spectra, out = real) or both (dir == 0), in the reverse pass
// order for the inverse (Sec. 2.1).
int wt_build(const fft3d_group_s* g, int dir, const void* const* rin, void* const* mid, void* const* rout,
             WtTable& t)
{
    t.nseg = 0;
    t.total = 0;
    const int stall = g->form == FFT3D_GROUP_WORK_TABLE_TEST_STALL;
    std::vector<int> prev(g->plans.size(), -1);
    int st = FFT3D_OK;
    if (dir <= 0)
        for (int pass = 0; pass < 3 && st == FFT3D_OK; ++pass) st = wt_add_pass(g, t, pass, -1, rin, rout, mid, prev);
    if (dir >= 0)
        for (int pass = 2; pass >= 0 && st == FFT3D_OK; --pass) st = wt_add_pass(g, t, pass, +1, rin, rout, mid, prev);
    if (stall)  // test form: the first dependency waits for one item more than exists
        for (int i = 0; i < t.nseg; ++i)
            if (t.seg[i].dep >= 0) {
                t.seg[i].need += 1;
                break;
            }
    return st;
}

int group_enqueue_wt(fft3d_group_s* g, int dir, const void* const* rin, void* const* mid, void* const* rout,
                     cudaStream_t s)
{
    WtTable t;
    const int st = wt_build(g, dir, rin, mid, rout, t);
    if (st != FFT3D_OK) return st;
    if (cudaMemsetAsync(g->d_ctr, 0, sizeof(WtCounters), s) != cudaSuccess) return FFT3D_ERR_CUDA;
    return launch_wt(t, g->d_ctr, s) == cudaSuccess ? FFT3D_OK : FFT3D_ERR_CUDA;
}

int group_enqueue(fft3d_group_s* g, int dir, const void* const* in, void* const* out, cudaStream_t s)
{
    if (cudaEventRecord(g->fork, s) != cudaSuccess) return FFT3D_ERR_CUDA;
    for (size_t i = 0; i < g->plans.size(); ++i) {
        if (cudaStreamWaitEvent(g->streams[i], g->fork, 0) != cudaSuccess) return FFT3D_ERR_CUDA;
        const int st = dir < 0 ? fft3d_r2c(g->plans[i], (const float*)in[i], out[i], g->streams[i])
                               : fft3d_c2r(g->plans[i], const_cast<void*>(in[i]), (float*)out[i], g->streams[i]);
        if (st != FFT3D_OK) return st;
        if (cudaEventRecord(g->joins[i], g->streams[i]) != cudaSuccess) return FFT3D_ERR_CUDA;
        if (cudaStreamWaitEvent(s, g->joins[i], 0) != cudaSuccess) return FFT3D_ERR_CUDA;
    }
    return FFT3D_OK;
}

// dir < 0: in -> mid (forward); dir > 0: mid -> out (inverse); dir == 0: both.
int group_run(fft3d_group_s* g, int dir, const void* const* in, void* const* mid, void* const* out, cudaStream_t s)
{
    if (g->form != FFT3D_GROUP_STREAMS) return group_enqueue_wt(g, dir, in, mid, out, s);
    int st = FFT3D_OK;
    if (dir <= 0) st = group_enqueue(g, -1, in, mid, s);
    if (st == FFT3D_OK && dir >= 0) st = group_enqueue(g, +1, const_cast<const void* const*>(mid), out, s);
    return st;
}

int group_exec(fft3d_group_s* g, int dir, const void* const* in, void* const* mid, void* const* out, cudaStream_t s)
{
    const size_t n = g->plans.size();
    for (size_t i = 0; i < n; ++i)
        if ((dir <= 0 && !in[i]) || !mid[i] || (dir >= 0 && !out[i])) return fail(FFT3D_ERR_INVALID_ARG);
    if (!s) {  // the legacy default stream cannot be captured: launch directly
        const int st = group_run(g, dir, in, mid, out, s);
        return st == FFT3D_OK ? FFT3D_OK : fail(st);
    }
    auto& gr = g->graphs[dir < 0 ? 0 : dir > 0 ? 1 : 2];
    bool same = gr.exec != nullptr && gr.mid.size() == n;
    for (size_t i = 0; same && i < n; ++i)
        same = (dir > 0 || gr.in[i] == in[i]) && gr.mid[i] == mid[i] && (dir < 0 || gr.out[i] == out[i]);
    if (!same) {
        if (gr.exec) cudaGraphExecDestroy(gr.exec);
        if (gr.graph) cudaGraphDestroy(gr.graph);
        gr.exec = nullptr;
        gr.graph = nullptr;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
        const int st = group_run(g, dir, in, mid, out, s);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s, &graph);
        if (st != FFT3D_OK || e != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            return fail(st != FFT3D_OK ? st : FFT3D_ERR_CUDA);
        }
        gr.graph = graph;
        if (cudaGraphInstantiate(&gr.exec, graph, 0) != cudaSuccess) {
            cudaGraphDestroy(graph);
            gr.graph = nullptr;
            return fail(FFT3D_ERR_CUDA);
        }
        gr.in.assign(in ? in : mid, (in ? in : mid) + n);
        gr.mid.assign(mid, mid + n);
        gr.out.assign(out ? out : mid, (out ? out : mid) + n);
    }
    return cudaGraphLaunch(gr.exec, s) == cudaSuccess ? FFT3D_OK : fail(FFT3D_ERR_CUDA);
}

}  // namespace

fft3d_group_handle fft3d_plan_group(const int* dims, const int* counts, int ngroups, int dtype)
{
    if (!dims || !counts || ngroups < 1 || ngroups > 64 || dtype == FFT3D_F64) {
        fail(FFT3D_ERR_INVALID_ARG);
        return nullptr;
    }
    fft3d_group_s* g = new (std::nothrow) fft3d_group_s();
    if (!g) {
        fail(FFT3D_ERR_ALLOC);
        return nullptr;
    }
    for (int i = 0; i < ngroups; ++i) {
        // the sizes of a group run concurrently on their own streams: their
        // plans keep the separate row and column passes (a persistent cluster
        // plane kernel, tuned alone, would hold every SM and serialise them)
        fft3d_handle p = fft3d_plan_variant(dims[3 * i], dims[3 * i + 1], dims[3 * i + 2], dtype, counts[i],
                                            FFT3D_FLAG_THREE_PASS);
        if (!p) {
            const int st = fft3d_last_error();
            group_free(g);
            fail(st);
            return nullptr;
        }
        g->plans.push_back(p);
        cudaStream_t st;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            group_free(g);
            fail(FFT3D_ERR_CUDA);
            return nullptr;
        }
        g->streams.push_back(st);
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            group_free(g);
            fail(FFT3D_ERR_CUDA);
            return nullptr;
        }
        g->joins.push_back(ev);
    }
    if (cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) != cudaSuccess) {
        group_free(g);
        fail(FFT3D_ERR_CUDA);
        return nullptr;
    }
    // the work-table form needs compiled item bodies for every size's passes
    g->wt_ok = dtype == FFT3D_F32;
    for (const fft3d_plan_s* p : g->plans) {
        if (!g->wt_ok) break;
        g->wt_ok = !(p->n2 & 1) && !(p->flags & FFT3D_FLAG_GENERIC) && p->ax0.spec && p->ax1.spec && p->ax2.spec;
        for (int dir : {-1, 1})
            g->wt_ok = g->wt_ok && wt_body_index(true, p->n2 / 2, dir, nullptr) >= 0 &&
                       wt_body_index(false, p->n1, dir, nullptr) >= 0 && wt_body_index(false, p->n0, dir, nullptr) >= 0;
    }
    WtTable probe;  // the table fits (segment count) -- operands are not needed to know that
    std::vector<void*> none(g->plans.size(), nullptr);
    if (g->wt_ok && wt_build(g, 0, const_cast<const void* const*>(none.data()), none.data(), none.data(), probe) != FFT3D_OK)
        g->wt_ok = false;
    if (g->wt_ok && cudaMalloc((void**)&g->d_ctr, sizeof(WtCounters)) != cudaSuccess) {
        group_free(g);
        fail(FFT3D_ERR_ALLOC);
        return nullptr;
    }
    // the streams form is the default: on GB300 it runs the 64^3 ... 192^3 x 4
    // group in 685-741 us per r2c + c2r against 853 us for the work table (whose
    // one register budget for every body holds it to 24 warps per SM)
    g->form = FFT3D_GROUP_STREAMS;
    return g;
}

fft3d_handle fft3d_group_plan_at(fft3d_group_handle g, int i)
{
    if (!g || i < 0 || i >= (int)g->plans.size()) {
        fail(FFT3D_ERR_INVALID_ARG);
        return nullptr;
    }
    return g->plans[(size_t)i];
}

int fft3d_group_r2c(fft3d_group_handle g, const float* const* in, void* const* out, void* stream)
{
    if (!g || !in || !out) return fail(FFT3D_ERR_INVALID_ARG);
    return group_exec(g, -1, reinterpret_cast<const void* const*>(in), out, nullptr, (cudaStream_t)stream);
}

int fft3d_group_c2r(fft3d_group_handle g, void* const* in, float* const* out, void* stream)
{
    if (!g || !in || !out) return fail(FFT3D_ERR_INVALID_ARG);
    return group_exec(g, +1, nullptr, in, reinterpret_cast<void* const*>(out), (cudaStream_t)stream);
}

int fft3d_group_r2c_c2r(fft3d_group_handle g, const float* const* in, void* const* mid, float* const* out,
                        void* stream)
{
    if (!g || !in || !mid || !out) return fail(FFT3D_ERR_INVALID_ARG);
    return group_exec(g, 0, reinterpret_cast<const void* const*>(in), mid, reinterpret_cast<void* const*>(out),
                      (cudaStream_t)stream);
}

int fft3d_group_launches(fft3d_group_handle g, int dir)
{
    if (!g) return fail(FFT3D_ERR_INVALID_ARG);
    if (g->form != FFT3D_GROUP_STREAMS) return 1;  // one work-table launch per call
    int n = 0;
    for (auto* p : g->plans) n += (dir <= 0 ? fft3d_launches_per_call(p, -1) : 0) + (dir >= 0 ? fft3d_launches_per_call(p, 1) : 0);
    return n;
}

int fft3d_group_set_form(fft3d_group_handle g, int form)
{
    if (!g || (form != FFT3D_GROUP_STREAMS && form != FFT3D_GROUP_WORK_TABLE &&
               form != FFT3D_GROUP_WORK_TABLE_TEST_STALL) ||
        (form != FFT3D_GROUP_STREAMS && !g->wt_ok))
        return fail(FFT3D_ERR_INVALID_ARG);
    if (form != g->form)
        for (auto& gr : g->graphs) {  // captured graphs hold the other form's launches
            if (gr.exec) cudaGraphExecDestroy(gr.exec);
            if (gr.graph) cudaGraphDestroy(gr.graph);
            gr = fft3d_group_s::Graph{};
        }
    g->form = form;
    return FFT3D_OK;
}

int fft3d_group_get_form(fft3d_group_handle g)
{
    if (!g) return -fail(FFT3D_ERR_INVALID_ARG);
    return g->form;
}

int fft3d_group_query_device_status(fft3d_group_handle g, void* stream)
{
    if (!g) return fail(FFT3D_ERR_INVALID_ARG);
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return fail(FFT3D_ERR_CUDA);
    int st = 0;
    if (g->d_ctr && cudaMemcpy(&st, &g->d_ctr->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(FFT3D_ERR_CUDA);
    for (auto* p : g->plans) {
        const int ps = fft3d_query_device_status(p, stream);
        if (ps != FFT3D_OK) return ps;
    }
    return (st & kStatusTimeout) ? fail(FFT3D_ERR_TIMEOUT) : FFT3D_OK;
}

void fft3d_group_destroy(fft3d_group_handle g)
{
    if (!g) return;
    cudaDeviceSynchronize();
    group_free(g);
}

int fft3d_set_profiling(fft3d_handle p, int enable)
{
    if (!p) return fail(FFT3D_ERR_INVALID_ARG);
    p->profiling = enable != 0;
    return FFT3D_OK;
}

int fft3d_profile_read(fft3d_handle p, double* ms, int* count, int n)
{
    if (!p || n < 0 || (n > 0 && (!ms || !count))) return fail(FFT3D_ERR_INVALID_ARG);
    for (int i = 0; i < n; ++i) {
        ms[i] = 0.0;
        count[i] = 0;
    }
    int st = FFT3D_OK;
    for (size_t i = 0; i < p->prof_used; ++i) {
        ProfRecord& r = p->prof[i];
        float t = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) {
            st = FFT3D_ERR_CUDA;
            continue;
        }
        if (r.pass < n) {
            ms[r.pass] += t;
            count[r.pass] += 1;
        }
    }
    p->prof_used = 0;
    return st == FFT3D_OK ? FFT3D_OK : fail(st);
}

const char* fft3d_pass_name(int pass)
{
    return (pass >= 0 && pass < PASS_COUNT) ? kPassNames[pass] : nullptr;
}

double fft3d_pass_bytes(fft3d_handle p, int pass)
{
    if (!p) return 0.0;
    const double B = p->batch, real = 4.0 * (double)p->N * B, cplx = 8.0 * (double)p->M * B;
    switch (pass) {
    case PASS_ROW_R2C:
    case PASS_ROW_C2R: return real + cplx;
    case PASS_N1_FWD:
    case PASS_N1_INV: return p->n1 > 1 ? 2.0 * cplx : 0.0;
    case PASS_N0_FWD:
    case PASS_N0_INV: return p->n0 > 1 ? 2.0 * cplx : 0.0;
    case PASS_SWAP01: return 2.0 * cplx;
    case PASS_PLANE_FWD:
    case PASS_PLANE_INV: return real + cplx;
    default: return 0.0;
    }
}

}  // extern "C"
