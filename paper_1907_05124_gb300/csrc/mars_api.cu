// Host runtime behind the C ABI of include/mars.h: contexts, instance ingest
// (validation, sweep order, level schedule, relabelling, device upload),
// solve orchestration and result readback. All arithmetic of the method runs
// in the kernels; this file moves data and makes decisions about launches.
#include "mars_host.h"

#include <cudaTypedefs.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <initializer_list>
#include <map>
#include <memory>
#include <numeric>
#include <string>
#include <vector>

using namespace mars;

// Levels a replica with start temperature t0 visits under p's schedule (an
// upper bound, counting a quench level).
double levels_bound(const mars_params* p, double t0)
{
    double L;
    if (p->schedule == MARS_SCHEDULE_GEOMETRIC)
        L = t0 > p->t_floor ? std::log(p->t_floor / t0) / std::log(p->cool_ratio) + 1.0 : 0.0;
    else
        L = t0 / p->c_step;
    return L + (p->quench ? 1.0 : 0.0);
}

// The labelled schedule variants' parameters; the paper's linear schedule
// needs none.
bool schedule_ok(const mars_params* p)
{
    if (p->schedule == MARS_SCHEDULE_LINEAR) return true;
    return p->schedule == MARS_SCHEDULE_GEOMETRIC && p->cool_ratio > 0.0 && p->cool_ratio < 1.0 &&
           p->t_floor > 0.0 && std::isfinite(p->t_floor);
}

const char* method_error(const mars_params* p)
{
    if (p->method == MARS_METHOD_MARS) return nullptr;
    if (p->method != MARS_METHOD_NMFA) return "unknown method";
    if (p->precision != MARS_FP32) return "NMFA runs with FP32 local fields only";
    if (p->quench) return "NMFA has no quench level";
    if (!(p->nmfa_alpha >= 0.0 && p->nmfa_alpha <= 1.0)) return "NMFA needs 0 <= nmfa_alpha <= 1";
    if (!(p->nmfa_sigma >= 0.0) || !std::isfinite(p->nmfa_sigma)) return "NMFA needs a finite nmfa_sigma >= 0";
    return nullptr;
}

void set_method(DevSolve& s, const mars_params* p)
{
    if (p->method != MARS_METHOD_NMFA) return;
    s.nmfa = 1;
    s.jacobi = 1;        // every spin's update from the same state
    s.fixed_sweeps = 1;  // one iteration per temperature level
    s.nmfa_alpha = (float)p->nmfa_alpha;
    s.nmfa_sigma = (float)p->nmfa_sigma;
}


int env_flag(const char* name, int dflt)
{
    const char* v = std::getenv(name);
    return v && *v ? std::atoi(v) : dflt;
}

int fail(mars_ctx* c, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}


int dev_alloc(mars_ctx* c, size_t bytes, DevMem* out)
{
    out->p = nullptr;
    out->bytes = 0;
    if (bytes == 0) return MARS_OK;
    if (c->fault_alloc_at > 0 && ++c->allocs == c->fault_alloc_at)
        return fail(c, MARS_ENOMEM, "device allocation %lld failed (injected by MARS_FAULT)",
                    (long long)c->allocs);
    if (c->budget && c->used + bytes > c->budget)
        return fail(c, MARS_ENOMEM, "HBM budget exceeded: %zu + %zu > %zu bytes", c->used, bytes,
                    c->budget);
    cudaError_t e = cudaMallocAsync(&out->p, bytes, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, MARS_ENOMEM, "device allocation of %zu bytes failed: %s", bytes,
                    cudaGetErrorString(e));
    }
    out->bytes = bytes;
    c->used += bytes;
    return MARS_OK;
}

int dev_alloc_on(mars_ctx* c, size_t bytes, DevMem* out, cudaStream_t st)
{
    out->p = nullptr;
    out->bytes = 0;
    if (bytes == 0) return MARS_OK;
    if (c->fault_alloc_at > 0 && ++c->allocs == c->fault_alloc_at)
        return fail(c, MARS_ENOMEM, "device allocation %lld failed (injected by MARS_FAULT)",
                    (long long)c->allocs);
    if (c->budget && c->used + bytes > c->budget)
        return fail(c, MARS_ENOMEM, "HBM budget exceeded: %zu + %zu > %zu bytes", c->used, bytes,
                    c->budget);
    cudaError_t e = cudaMallocAsync(&out->p, bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, MARS_ENOMEM, "device allocation of %zu bytes failed: %s", bytes,
                    cudaGetErrorString(e));
    }
    out->bytes = bytes;
    c->used += bytes;
    return MARS_OK;
}

void dev_free_on(mars_ctx* c, DevMem* m, cudaStream_t st)
{
    if (m->p) {
        cudaFreeAsync(m->p, st);
        c->used -= m->bytes;
    }
    m->p = nullptr;
    m->bytes = 0;
}

void dev_free(mars_ctx* c, DevMem* m)
{
    if (m->p) {
        cudaFreeAsync(m->p, c->stream);
        c->used -= m->bytes;
    }
    m->p = nullptr;
    m->bytes = 0;
}


template <typename T>
int upload(mars_ctx* c, Instance* in, const std::vector<T>& v, const T** out)
{
    *out = nullptr;
    if (v.empty()) return MARS_OK;
    DevMem m;
    int rc = dev_alloc(c, v.size() * sizeof(T), &m);
    if (rc) return rc;
    in->mem.push_back(m);
    MARS_CUDA(c, cudaMemcpyAsync(m.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice,
                                 c->stream));
    *out = (const T*)m.p;
    return MARS_OK;
}

// Copy `count` elements from host or device memory into a host vector.
template <typename T>
int fetch(mars_ctx* c, const void* src, size_t count, bool device, std::vector<T>* out)
{
    out->resize(count);
    if (count == 0) return MARS_OK;
    if (device) {
        MARS_CUDA(c, cudaMemcpyAsync(out->data(), src, count * sizeof(T), cudaMemcpyDeviceToHost,
                                     c->stream));
        MARS_CUDA(c, cudaStreamSynchronize(c->stream));
    } else {
        std::memcpy(out->data(), src, count * sizeof(T));
    }
    return MARS_OK;
}

int fetch_values(mars_ctx* c, const void* src, size_t count, int32_t dt, bool device,
                 std::vector<double>* out)
{
    int rc;
    switch (dt) {
    case MARS_I8: {
        std::vector<int8_t> v;
        if ((rc = fetch(c, src, count, device, &v))) return rc;
        out->assign(v.begin(), v.end());
        return MARS_OK;
    }
    case MARS_F32: {
        std::vector<float> v;
        if ((rc = fetch(c, src, count, device, &v))) return rc;
        out->assign(v.begin(), v.end());
        return MARS_OK;
    }
    case MARS_F64:
        return fetch(c, src, count, device, out);
    default:
        return fail(c, MARS_EINVAL, "unknown value type %d", dt);
    }
}

int check_order(mars_ctx* c, const int32_t* order, int32_t n, std::vector<int32_t>* out)
{
    out->resize(n);
    if (!order) {
        std::iota(out->begin(), out->end(), 0);
        return MARS_OK;
    }
    std::vector<char> seen(n, 0);
    for (int32_t q = 0; q < n; ++q) {
        const int32_t v = order[q];
        if (v < 0 || v >= n || seen[v]) return fail(c, MARS_EINVAL, "order is not a permutation");
        seen[v] = 1;
        (*out)[q] = v;
    }
    return MARS_OK;
}

bool is_small_int(double v, double lim) { return v == std::floor(v) && std::fabs(v) <= lim; }

// Span of the exact energy accumulator (exact_sum.cuh): e0 is the weight of
// the last mantissa bit of the smallest non-zero term; the sum of `terms`
// terms of at most max|v| must stay below 2^(e0 + 220).
void exact_span(const std::vector<double>& vals, const std::vector<double>& h, int64_t terms,
                DevInstance* d)
{
    int lo = INT32_MAX, hi = INT32_MIN;
    auto visit = [&](double v) {
        if (v == 0.0) return;
        int e;
        std::frexp(std::fabs(v), &e);   // |v| = f 2^e, 0.5 <= f < 1
        lo = std::min(lo, e - 53);       // weight of the last mantissa bit
        hi = std::max(hi, e);            // |v| < 2^e
    };
    for (double v : vals) visit(v);
    for (double v : h) visit(v);
    if (lo == INT32_MAX) { d->exact_ok = 1; d->exact_e0 = 0; return; }
    int grow = 0;
    while ((int64_t)1 << grow < terms + 1 && grow < 62) ++grow;
    d->exact_e0 = lo;
    d->exact_ok = (hi + grow - lo) <= 220 && lo >= -1126;
}

int finish_register(mars_ctx* c, std::unique_ptr<Instance> in, int32_t* inst)
{
    in->info.device_bytes = 0;
    for (auto& m : in->mem) in->info.device_bytes += (int64_t)m.bytes;
    const int32_t id = c->next_id++;
    c->insts[id] = std::move(in);
    if (inst) *inst = id;
    return MARS_OK;
}

// Frees the device buffers of an instance whose registration failed.
struct InstGuard {
    mars_ctx* c;
    Instance* in;
    bool done = false;
    ~InstGuard()
    {
        if (!done)
            for (auto& m : in->mem) dev_free(c, &m);
    }
};

Instance* find(mars_ctx* c, int32_t id)
{
    auto it = c->insts.find(id);
    return it == c->insts.end() ? nullptr : it->second.get();
}


// Round-to-nearest-even FP32 -> BF16 bits (host side, for uploads).
uint16_t float_to_bf16_bits(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, sizeof u);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;  // NaN
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

// Host-side fault injection for tests (MARS_FAULT, a comma-separated list):
// "alloc:K" fails the context's K-th device allocation, "flag" withholds
// mars_device_check's flag. Unknown items are ignored.
void parse_faults(mars_ctx* c, const char* spec)
{
    if (!spec) return;
    std::string all(spec);
    size_t pos = 0;
    while (pos <= all.size()) {
        const size_t end = std::min(all.find(',', pos), all.size());
        const std::string item = all.substr(pos, end - pos);
        if (item.rfind("alloc:", 0) == 0) c->fault_alloc_at = std::atoll(item.c_str() + 6);
        if (item == "flag") c->fault_flag = true;
        pos = end + 1;
    }
}

// Accessors for mars_noalloc.cu.
int noalloc_view(mars_ctx* c, int32_t id, NoallocView* v)
{
    if (!c || !v) return MARS_EINVAL;
    Instance* in = find(c, id);
    if (!in) return fail(c, MARS_ENOTFOUND, "unknown instance %d", id);
    v->device = c->device;
    v->stream = c->stream;
    v->inst = &in->dev;
    v->scratch_base = &c->noalloc_base;
    v->total_weight = in->info.total_weight;
    v->energy_err_bound = (in->dev.integer || in->dev.exact_ok)
                              ? 0.0
                              : std::ldexp(in->abs_weight, -53) * (double)(in->info.nnz / 2 + in->dev.n);
    return MARS_OK;
}

int noalloc_fail(mars_ctx* c, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

extern "C" {

int mars_create(mars_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream)
{
    if (!out) return MARS_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return MARS_EDEVICE;
    }
    auto c = std::make_unique<mars_ctx>();
    c->device = device;
    c->budget = hbm_budget_bytes;
    DeviceGuard g(device);
    if (cudaFree(nullptr) != cudaSuccess) return MARS_EDEVICE;  // create the primary context
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return MARS_EDEVICE;
        c->own_stream = true;
    }
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    parse_faults(c.get(), std::getenv("MARS_FAULT"));
    if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess ||
        cudaEventCreate(&c->ev2) != cudaSuccess || cudaEventCreate(&c->ev3) != cudaSuccess)
        return MARS_EDEVICE;
    *out = c.release();
    return MARS_OK;
}

void mars_destroy(mars_ctx* c)
{
    if (!c) return;
    {
        DeviceGuard g(c->device);
        serve_release(c);
        for (auto& kv : c->insts)
            for (auto& m : kv.second->mem) dev_free(c, &m);
        c->insts.clear();
        cudaStreamSynchronize(c->stream);
        if (c->ev0) cudaEventDestroy(c->ev0);
        if (c->ev1) cudaEventDestroy(c->ev1);
        if (c->ev2) cudaEventDestroy(c->ev2);
        if (c->ev3) cudaEventDestroy(c->ev3);
        if (c->check_flag) cudaFreeHost(c->check_flag);
        if (c->check_status) cudaFree(c->check_status);
        if (c->own_stream) cudaStreamDestroy(c->stream);
    }
    delete c;
}

const char* mars_last_error(mars_ctx* c) { return c ? c->err.c_str() : "null context"; }

void mars_params_default(mars_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->replicas = 1;
    p->t_min = 0.0;
    p->t_max = 1.0;
    p->c_step = 1.0;
    p->d_min = 1e-4;
    p->k_max = 1000;
    p->update = MARS_UPDATE_GS;
    p->precision = MARS_FP32;
    p->method = MARS_METHOD_MARS;
    p->nmfa_alpha = 0.5;
    p->nmfa_sigma = 0.0;
}

int mars_instance_dense(mars_ctx* c, int32_t n, const void* J, int32_t jt, const double* h,
                        const int32_t* order, uint32_t flags, int32_t* inst)
{
    if (!c) return MARS_EINVAL;
    if (n <= 0 || !J) return fail(c, MARS_EINVAL, "dense instance needs n > 0 and J");
    if ((int64_t)n * n > (int64_t)1 << 31) return fail(c, MARS_EINVAL, "n too large for dense J");
    DeviceGuard g(c->device);
    const bool devp = flags & MARS_DEVICE_PTR;
    std::vector<double> Jh, hh;
    int rc = fetch_values(c, J, (size_t)n * n, jt, devp, &Jh);
    if (rc) return rc;
    if (h && (rc = fetch(c, h, (size_t)n, false, &hh))) return rc;
    bool integer = true;
    double wsum = 0.0, aw = 0.0;
    long long wint = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (Jh[(size_t)i * n + i] != 0.0)
            return fail(c, MARS_EINVAL, "J has a non-zero diagonal entry at %d", i);
        for (int32_t j = i + 1; j < n; ++j) {
            const double a = Jh[(size_t)i * n + j], b = Jh[(size_t)j * n + i];
            if (!std::isfinite(a) || a != b)
                return fail(c, MARS_EINVAL, "J is not symmetric and finite at (%d,%d)", i, j);
            integer = integer && is_small_int(a, 127.0);
            wsum += a;
            aw += std::fabs(a);
            if (integer) wint += (long long)a;
        }
    }
    for (double v : hh) {
        if (!std::isfinite(v)) return fail(c, MARS_EINVAL, "h has a non-finite entry");
        integer = integer && is_small_int(v, 16777216.0);
        aw += std::fabs(v);
    }
    auto in = std::make_unique<Instance>();
    InstGuard guard{c, in.get()};
    if ((rc = check_order(c, order, n, &in->order))) return rc;
    const std::vector<int32_t>& o = in->order;  // new label a is caller spin o[a]
    std::vector<float> Jf((size_t)n * n);
    std::vector<int8_t> Ji;
    std::vector<double> Jd;
    if (integer) Ji.resize((size_t)n * n); else Jd.resize((size_t)n * n);
    for (int32_t a = 0; a < n; ++a)
        for (int32_t b = 0; b < n; ++b) {
            const double v = Jh[(size_t)o[a] * n + o[b]];
            Jf[(size_t)a * n + b] = (float)v;
            if (integer) Ji[(size_t)a * n + b] = (int8_t)v; else Jd[(size_t)a * n + b] = v;
        }
    std::vector<float> hf;
    std::vector<double> hd;
    if (!hh.empty()) {
        hf.resize(n);
        hd.resize(n);
        for (int32_t a = 0; a < n; ++a) { hf[a] = (float)hh[o[a]]; hd[a] = hh[o[a]]; }
    }
    // Tensor-core operands: BF16 J padded to whole 128-spin panels, the
    // panels' FP32 diagonal blocks for the in-panel sequential updates, and
    // the FP32 blocks J[p][p+1] through which a chain feeds the next panel.
    const int32_t n_pad = (n + 127) / 128 * 128;
    std::vector<uint16_t> Jb((size_t)n_pad * n_pad, 0);
    std::vector<float> Jdiag((size_t)n_pad * 128, 0.f), Jsup((size_t)n_pad * 128, 0.f);
    for (int32_t a = 0; a < n; ++a)
        for (int32_t b = 0; b < n; ++b) {
            const float v = Jf[(size_t)a * n + b];
            Jb[(size_t)a * n_pad + b] = float_to_bf16_bits(v);
            if (a / 128 == b / 128)
                Jdiag[((size_t)(a / 128) * 128 + a % 128) * 128 + b % 128] = v;
            else if (b / 128 == a / 128 + 1)
                Jsup[((size_t)(a / 128) * 128 + a % 128) * 128 + b % 128] = v;
        }
    // E4M3 copy for FP8 descents, when every coupling is exact in E4M3
    // (integers up to 16, and coarser ones up to 448).
    std::vector<uint8_t> J8;
    if (integer) {
        J8.assign((size_t)n_pad * n_pad, 0);
        bool exact = true;
        for (int32_t a = 0; a < n && exact; ++a)
            for (int32_t b = 0; b < n; ++b) {
                const float v = Jf[(size_t)a * n + b];
                const __nv_fp8_e4m3 q(v);
                if (float(q) != v) {
                    exact = false;
                    break;
                }
                J8[(size_t)a * n_pad + b] = (uint8_t)q.__x;
            }
        if (!exact) J8.clear();
    }
    DevInstance& d = in->dev;
    d.n = n;
    d.dense = 1;
    d.nnz = (int64_t)n * (n - 1);
    d.nlev = n;
    d.integer = integer;
    d.n_pad = n_pad;
    if (!integer) exact_span(Jh, hh, (int64_t)n * (n - 1) / 2 + n, &d);
    {
        const uint16_t* jb = nullptr;
        if ((rc = upload(c, in.get(), Jb, &jb))) return rc;
        d.Jbf = (const __nv_bfloat16*)jb;
        if ((rc = upload(c, in.get(), Jdiag, &d.Jdiag))) return rc;
        if ((rc = upload(c, in.get(), Jsup, &d.Jsup))) return rc;
        if (!J8.empty() && (rc = upload(c, in.get(), J8, &d.J8))) return rc;
    }
    if ((rc = upload(c, in.get(), Jf, &d.Jf))) return rc;
    if ((rc = upload(c, in.get(), Ji, &d.J_i8))) return rc;
    if ((rc = upload(c, in.get(), Jd, &d.J_f64))) return rc;
    if ((rc = upload(c, in.get(), hf, &d.h))) return rc;
    if ((rc = upload(c, in.get(), hd, &d.h_f64))) return rc;
    if ((rc = upload(c, in.get(), o, &d.new2old))) return rc;
    {
        // NMFA's field normalisation, 1 / sqrt(h_a^2 + sum_b J_ab^2), in FP64
        std::vector<float> inv(n);
        for (int32_t a = 0; a < n; ++a) {
            double q = 0.0;
            for (int32_t b = 0; b < n; ++b) {
                const double v = Jh[(size_t)o[a] * n + o[b]];
                q += v * v;
            }
            if (!hh.empty()) q += hh[o[a]] * hh[o[a]];
            inv[a] = q > 0.0 ? (float)(1.0 / std::sqrt(q)) : 0.f;
        }
        if ((rc = upload(c, in.get(), inv, &d.inv_norm))) return rc;
    }
    MARS_CUDA(c, cudaStreamSynchronize(c->stream));
    guard.done = true;
    in->info.n = n;
    in->info.dense = 1;
    in->info.nnz = d.nnz;
    in->info.levels = n;
    in->info.integer = integer;
    in->info.total_weight = integer ? (double)wint : wsum;
    in->abs_weight = aw;
    return finish_register(c, std::move(in), inst);
}

int mars_instance_csr(mars_ctx* c, int32_t n, int64_t nnz, const int32_t* row_ptr,
                      const int32_t* col, const void* val, int32_t vt, const double* h,
                      const int32_t* order, uint32_t flags, int32_t* inst)
{
    if (!c) return MARS_EINVAL;
    if (n <= 0 || nnz < 0 || nnz > INT32_MAX || !row_ptr || (nnz > 0 && (!col || !val)))
        return fail(c, MARS_EINVAL, "CSR instance needs n > 0, 0 <= nnz < 2^31 and arrays");
    DeviceGuard g(c->device);
    const bool devp = flags & MARS_DEVICE_PTR;
    std::vector<int32_t> rp, cl;
    std::vector<double> vl, hh;
    int rc;
    if ((rc = fetch(c, row_ptr, (size_t)n + 1, devp, &rp))) return rc;
    if ((rc = fetch(c, col, (size_t)nnz, devp, &cl))) return rc;
    if ((rc = fetch_values(c, val, (size_t)nnz, vt, devp, &vl))) return rc;
    if (h && (rc = fetch(c, h, (size_t)n, false, &hh))) return rc;
    if (rp[0] != 0 || rp[n] != nnz) return fail(c, MARS_EINVAL, "row_ptr must run from 0 to nnz");
    for (int32_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) return fail(c, MARS_EINVAL, "row_ptr decreases at row %d", i);
    // Rows with columns sorted (stable on a copy) to check duplicates and symmetry.
    std::vector<int32_t> sc(cl);
    std::vector<double> sv(vl);
    {
        std::vector<int64_t> idx;
        for (int32_t i = 0; i < n; ++i) {
            const int32_t e0 = rp[i], e1 = rp[i + 1];
            idx.resize(e1 - e0);
            std::iota(idx.begin(), idx.end(), (int64_t)e0);
            std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return cl[a] < cl[b]; });
            for (int32_t q = 0; q < e1 - e0; ++q) { sc[e0 + q] = cl[idx[q]]; sv[e0 + q] = vl[idx[q]]; }
            for (int32_t e = e0; e < e1; ++e) {
                if (sc[e] < 0 || sc[e] >= n) return fail(c, MARS_EINVAL, "column out of range in row %d", i);
                if (sc[e] == i) return fail(c, MARS_EINVAL, "diagonal entry in row %d", i);
                if (e > e0 && sc[e] == sc[e - 1]) return fail(c, MARS_EINVAL, "repeated column in row %d", i);
                if (!std::isfinite(sv[e])) return fail(c, MARS_EINVAL, "non-finite value in row %d", i);
            }
        }
    }
    bool integer = true;
    double wsum = 0.0, aw = 0.0;
    long long wint = 0;
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int32_t j = sc[e];
            const auto b = sc.begin() + rp[j], en = sc.begin() + rp[j + 1];
            const auto it = std::lower_bound(b, en, i);
            if (it == en || *it != i || sv[it - sc.begin()] != sv[e])
                return fail(c, MARS_EINVAL, "couplings are not symmetric at (%d,%d)", i, j);
            if (j > i) {
                integer = integer && is_small_int(sv[e], 127.0);
                wsum += sv[e];
                aw += std::fabs(sv[e]);
                if (integer) wint += (long long)sv[e];
            }
        }
    }
    for (double v : hh) {
        if (!std::isfinite(v)) return fail(c, MARS_EINVAL, "h has a non-finite entry");
        integer = integer && is_small_int(v, 16777216.0);
        aw += std::fabs(v);
    }
    auto in = std::make_unique<Instance>();
    InstGuard guard{c, in.get()};
    // Visiting order: the caller's, or greedy colour classes in turn.
    if (order) {
        if ((rc = check_order(c, order, n, &in->order))) return rc;
    } else {
        std::vector<int32_t> colour(n, -1);
        std::vector<int32_t> mark;
        for (int32_t i = 0; i < n; ++i) {
            mark.assign(rp[i + 1] - rp[i] + 2, 0);
            for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
                const int32_t cj = colour[sc[e]];
                if (cj >= 0 && cj < (int32_t)mark.size()) mark[cj] = 1;
            }
            int32_t cc = 0;
            while (mark[cc]) ++cc;
            colour[i] = cc;
        }
        in->order.resize(n);
        std::iota(in->order.begin(), in->order.end(), 0);
        std::stable_sort(in->order.begin(), in->order.end(),
                         [&](int32_t a, int32_t b) { return colour[a] < colour[b]; });
    }
    // Level schedule of the sequential sweep in that order.
    std::vector<int32_t> pos(n), level(n, 0);
    for (int32_t q = 0; q < n; ++q) pos[in->order[q]] = q;
    int32_t nlev = 0;
    for (int32_t q = 0; q < n; ++q) {
        const int32_t v = in->order[q];
        int32_t lv = 0;
        for (int32_t e = rp[v]; e < rp[v + 1]; ++e)
            if (pos[sc[e]] < q) lv = std::max(lv, level[sc[e]] + 1);
        level[v] = lv;
        nlev = std::max(nlev, lv + 1);
    }
    // New labels: by level, then by degree (descending) so that the 32-row
    // slices of the ELL copy are nearly uniform, then by visiting position.
    // Spins of one level share no coupling, so their relative order is free.
    std::vector<int32_t> new2old(n), old2new(n), lvl_start(nlev + 1, 0);
    std::iota(new2old.begin(), new2old.end(), 0);
    std::stable_sort(new2old.begin(), new2old.end(), [&](int32_t a, int32_t b) {
        if (level[a] != level[b]) return level[a] < level[b];
        const int32_t da = rp[a + 1] - rp[a], db = rp[b + 1] - rp[b];
        if (da != db) return da > db;
        return pos[a] < pos[b];
    });
    for (int32_t a = 0; a < n; ++a) { old2new[new2old[a]] = a; lvl_start[level[new2old[a]] + 1]++; }
    for (int32_t l = 0; l < nlev; ++l) lvl_start[l + 1] += lvl_start[l];
    // CSR over new labels with columns sorted.
    std::vector<int32_t> nrp(n + 1, 0), ncol(nnz);
    std::vector<float> nval(nnz);
    std::vector<int8_t> nval_i8(integer ? nnz : 0);
    std::vector<double> nval_f64(nnz);
    std::vector<std::pair<int32_t, double>> row;
    for (int32_t a = 0; a < n; ++a) {
        const int32_t o = new2old[a];
        row.clear();
        for (int32_t e = rp[o]; e < rp[o + 1]; ++e) row.emplace_back(old2new[sc[e]], sv[e]);
        std::sort(row.begin(), row.end());
        nrp[a + 1] = nrp[a] + (int32_t)row.size();
        for (size_t q = 0; q < row.size(); ++q) {
            const int32_t e = nrp[a] + (int32_t)q;
            ncol[e] = row[q].first;
            nval[e] = (float)row[q].second;
            nval_f64[e] = row[q].second;
            if (integer) nval_i8[e] = (int8_t)row[q].second;
        }
    }
    // Sliced-ELL copy: per level, 32 consecutive new labels per slice, entries
    // slot-major and padded to the slice's largest degree with the dummy spin n.
    bool pm1 = integer;
    for (int64_t e = 0; e < nnz && pm1; ++e) pm1 = nval_f64[e] == 1.0 || nval_f64[e] == -1.0;
    std::vector<int32_t> lvl_slice(nlev + 1, 0);
    std::vector<int32_t> slice_words;  // row0, rows, degree, offset per slice
    std::vector<uint32_t> sell_pm1;
    std::vector<uint16_t> sell16;      // the same as halfwords when every column fits 15 bits
    const bool half = pm1 && n < 32768;
    std::vector<int32_t> sell_gen;     // (column, float bits) pairs
    int64_t sell_len = 0;
    for (int32_t l = 0; l < nlev; ++l) {
        for (int32_t r0 = lvl_start[l]; r0 < lvl_start[l + 1]; r0 += 32) {
            const int32_t rows = std::min(32, lvl_start[l + 1] - r0);
            int32_t deg = 0;
            for (int32_t q = 0; q < rows; ++q) deg = std::max(deg, nrp[r0 + q + 1] - nrp[r0 + q]);
            slice_words.insert(slice_words.end(), {r0, rows, deg, (int32_t)sell_len});
            for (int32_t t = 0; t < deg; ++t) {
                for (int32_t q = 0; q < 32; ++q) {
                    int32_t cidx = n;
                    double w = 0.0;
                    if (q < rows && t < nrp[r0 + q + 1] - nrp[r0 + q]) {
                        cidx = ncol[nrp[r0 + q] + t];
                        w = nval_f64[nrp[r0 + q] + t];
                    }
                    if (pm1) {
                        sell_pm1.push_back((uint32_t)cidx | (w < 0 ? 0x80000000u : 0u));
                        if (half) sell16.push_back((uint16_t)((uint32_t)cidx | (w < 0 ? 0x8000u : 0u)));
                    } else {
                        const float wf = (float)w;
                        int32_t bits;
                        std::memcpy(&bits, &wf, sizeof bits);
                        sell_gen.push_back(cidx);
                        sell_gen.push_back(bits);
                    }
                }
            }
            sell_len += (int64_t)deg * 32;
            if (sell_len > INT32_MAX) return fail(c, MARS_EINVAL, "padded coupling table too large");
        }
        lvl_slice[l + 1] = (int32_t)(slice_words.size() / 4);
    }
    std::vector<float> hf;
    std::vector<double> hd;
    if (!hh.empty()) {
        hf.resize(n);
        hd.resize(n);
        for (int32_t a = 0; a < n; ++a) { hf[a] = (float)hh[new2old[a]]; hd[a] = hh[new2old[a]]; }
    }
    DevInstance& d = in->dev;
    {
        const int32_t* sw = nullptr;
        if ((rc = upload(c, in.get(), slice_words, &sw))) return rc;
        d.slices = (const int4*)sw;
        if ((rc = upload(c, in.get(), lvl_slice, &d.lvl_slice))) return rc;
        if ((rc = upload(c, in.get(), sell_pm1, &d.sell_pm1))) return rc;
        if ((rc = upload(c, in.get(), sell16, &d.sell16))) return rc;
        d.nslices = (int32_t)(slice_words.size() / 4);
        d.sell_len = sell_len;
        int32_t deg0 = rp[1] - rp[0];
        for (int32_t i = 1; i < n && deg0 >= 0; ++i)
            if (rp[i + 1] - rp[i] != deg0) deg0 = -1;
        d.regular_deg = deg0 > 0 ? deg0 : 0;
        const int32_t* sg = nullptr;
        if ((rc = upload(c, in.get(), sell_gen, &sg))) return rc;
        d.sell_gen = (const int2*)sg;
    }
    d.n = n;
    d.dense = 0;
    d.nnz = nnz;
    if (!integer) exact_span(nval_f64, hh, nnz / 2 + n, &d);
    d.nlev = nlev;
    d.integer = integer;
    if ((rc = upload(c, in.get(), nrp, &d.row_ptr))) return rc;
    if ((rc = upload(c, in.get(), ncol, &d.col))) return rc;
    if ((rc = upload(c, in.get(), nval, &d.val))) return rc;
    if ((rc = upload(c, in.get(), nval_i8, &d.val_i8))) return rc;
    if ((rc = upload(c, in.get(), nval_f64, &d.val_f64))) return rc;
    if ((rc = upload(c, in.get(), lvl_start, &d.lvl_start))) return rc;
    if ((rc = upload(c, in.get(), hf, &d.h))) return rc;
    if ((rc = upload(c, in.get(), hd, &d.h_f64))) return rc;
    if ((rc = upload(c, in.get(), new2old, &d.new2old))) return rc;
    {
        // NMFA's field normalisation, 1 / sqrt(h_i^2 + sum_j J_ij^2), in FP64
        std::vector<float> inv(n);
        for (int32_t a = 0; a < n; ++a) {
            double q = 0.0;
            for (int32_t e = nrp[a]; e < nrp[a + 1]; ++e) q += nval_f64[e] * nval_f64[e];
            if (!hh.empty()) q += hh[new2old[a]] * hh[new2old[a]];
            inv[a] = q > 0.0 ? (float)(1.0 / std::sqrt(q)) : 0.f;
        }
        if ((rc = upload(c, in.get(), inv, &d.inv_norm))) return rc;
    }
    MARS_CUDA(c, cudaStreamSynchronize(c->stream));
    guard.done = true;
    in->info.n = n;
    in->info.dense = 0;
    in->info.nnz = nnz;
    in->info.levels = nlev;
    in->info.integer = integer;
    in->info.total_weight = integer ? (double)wint : wsum;
    in->abs_weight = aw;
    return finish_register(c, std::move(in), inst);
}

int mars_instance_free(mars_ctx* c, int32_t id)
{
    if (!c) return MARS_EINVAL;
    auto it = c->insts.find(id);
    if (it == c->insts.end()) return fail(c, MARS_ENOTFOUND, "unknown instance %d", id);
    DeviceGuard g(c->device);
    for (auto& m : it->second->mem) dev_free(c, &m);
    c->insts.erase(it);
    return MARS_OK;
}

int mars_instance_get_info(mars_ctx* c, int32_t id, mars_instance_info* info)
{
    if (!c || !info) return MARS_EINVAL;
    Instance* in = find(c, id);
    if (!in) return fail(c, MARS_ENOTFOUND, "unknown instance %d", id);
    *info = in->info;
    return MARS_OK;
}

int mars_instance_order(mars_ctx* c, int32_t id, int32_t* order_out)
{
    if (!c || !order_out) return MARS_EINVAL;
    Instance* in = find(c, id);
    if (!in) return fail(c, MARS_ENOTFOUND, "unknown instance %d", id);
    std::memcpy(order_out, in->order.data(), in->order.size() * sizeof(int32_t));
    return MARS_OK;
}

int mars_solve(mars_ctx* c, int32_t id, const mars_params* p, int8_t* best_spins,
               const mars_outputs* outs, mars_result* result)
{
    if (!c || !p) return MARS_EINVAL;
    Instance* in = find(c, id);
    if (!in) return fail(c, MARS_ENOTFOUND, "unknown instance %d", id);
    const int32_t R = p->replicas, n = in->dev.n;
    if (R < 1) return fail(c, MARS_EINVAL, "replicas must be >= 1");
    if (!std::isfinite(p->t_min) || !std::isfinite(p->t_max) || p->t_min > p->t_max)
        return fail(c, MARS_EINVAL, "need finite t_min <= t_max");
    if (!(p->c_step > 0.0) || !std::isfinite(p->c_step)) return fail(c, MARS_EINVAL, "c_step must be > 0");
    if (!schedule_ok(p)) return fail(c, MARS_EINVAL, "bad schedule (geometric: 0 < cool_ratio < 1, t_floor > 0)");
    if (levels_bound(p, p->t_max) > kMaxLevels)
        return fail(c, MARS_EINVAL, "t_max needs more than %.0f temperature levels", kMaxLevels);
    if (!(p->d_min >= 0.0)) return fail(c, MARS_EINVAL, "d_min must be >= 0");
    if (p->k_max < 1 || p->fixed_sweeps < 0) return fail(c, MARS_EINVAL, "k_max >= 1, fixed_sweeps >= 0");
    if (p->update != MARS_UPDATE_GS && p->update != MARS_UPDATE_JACOBI)
        return fail(c, MARS_EINVAL, "unknown update rule %d", p->update);
    if (const char* e = method_error(p)) return fail(c, MARS_EINVAL, "%s", e);
    const bool tc = p->precision == MARS_BF16 || p->precision == MARS_FP8;
    if (p->precision != MARS_FP32 && !(tc && in->dev.dense && p->update == MARS_UPDATE_GS))
        return fail(c, MARS_EINVAL, "precision %d is not available for this instance and update rule",
                    p->precision);
    if (p->precision == MARS_FP8 && !in->dev.J8)
        return fail(c, MARS_EINVAL, "FP8 needs integer couplings exactly representable in E4M3");
    if ((size_t)R * n > ((size_t)1 << 40)) return fail(c, MARS_EINVAL, "R*n too large");
    DeviceGuard g(c->device);
    cudaStream_t st = c->stream;
    const bool pdev = p->flags & MARS_DEVICE_PTR;
    const bool odev = outs && (outs->flags & MARS_DEVICE_PTR);
    Scratch S(c);
    int rc;
    int64_t launches = 0;  // kernels this solve launches
    DevSolve s;
    s.R = R;
    s.seed = p->seed;
    s.stream = p->stream;
    s.c_step = p->c_step;
    s.d_min = (float)p->d_min;
    s.k_max = p->k_max;
    s.fixed_sweeps = p->fixed_sweeps;
    set_schedule(s, p);
    s.jacobi = p->update == MARS_UPDATE_JACOBI;
    set_method(s, p);
    // start temperatures
    float* t0 = nullptr;
    if ((rc = S.get(R, &t0))) return rc;
    std::vector<float> t0h(R);
    if (p->t0) {
        if (pdev) {
            MARS_CUDA(c, cudaMemcpyAsync(t0, p->t0, R * sizeof(float), cudaMemcpyDeviceToDevice, st));
            MARS_CUDA(c, cudaMemcpyAsync(t0h.data(), p->t0, R * sizeof(float), cudaMemcpyDeviceToHost, st));
        } else {
            std::memcpy(t0h.data(), p->t0, R * sizeof(float));
            MARS_CUDA(c, cudaMemcpyAsync(t0, t0h.data(), R * sizeof(float), cudaMemcpyHostToDevice, st));
        }
    } else {
        MARS_CUDA(c, launch_draw(p->seed, p->stream, 0, R, 0, p->t_min, p->t_max, nullptr, t0, st));
        MARS_CUDA(c, cudaMemcpyAsync(t0h.data(), t0, R * sizeof(float), cudaMemcpyDeviceToHost, st));
        ++launches;
    }
    for (float v : t0h)
        if (!std::isfinite(v) || levels_bound(p, v) > kMaxLevels)
            return fail(c, MARS_EINVAL, "start temperatures must be finite with t0 / c_step <= %.0f",
                        kMaxLevels);
    s.t0 = t0;
    if (p->m0) {
        if (pdev) {
            s.m0 = p->m0;
        } else {
            float* m0 = nullptr;
            if ((rc = S.get((size_t)R * n, &m0))) return rc;
            MARS_CUDA(c, cudaMemcpyAsync(m0, p->m0, (size_t)R * n * sizeof(float),
                                         cudaMemcpyHostToDevice, st));
            s.m0 = m0;
        }
    }
    // per-replica outputs
    if ((rc = S.get((size_t)R * n, &s.sigma))) return rc;
    if ((rc = S.get(R, &s.energy))) return rc;
    if ((rc = S.get(R, &s.energy_i64))) return rc;
    if ((rc = S.get(R, &s.sweeps))) return rc;
    if ((rc = S.get(R, &s.levels))) return rc;
    if ((rc = S.get(R, &s.capped))) return rc;
    if ((rc = S.get(2, &s.work_counter))) return rc;
    s.status = s.work_counter + 1;
    MARS_CUDA(c, cudaMemsetAsync(s.work_counter, 0, 2 * sizeof(int32_t), st));
    if (outs && outs->m_final) {
        if (odev) {
            s.m_final = outs->m_final;
        } else if ((rc = S.get((size_t)R * n, &s.m_final))) {
            return rc;
        }
    }
    DevResult* dres = nullptr;
    int8_t* dbest = nullptr;
    if ((rc = S.get(1, &dres))) return rc;
    if ((rc = S.get(n, &dbest))) return rc;
    // Schedule: replicas by start temperature, longest descents first.
    MARS_CUDA(c, cudaStreamSynchronize(st));
    SparsePlan sp;
    DensePlan dp;
    WidePlan wp;
    bool wide = false;
    int rt = 1;
    if (in->dev.dense && !tc) {
        dp = plan_dense(in->dev, R, s.jacobi, c->device);
        if (dp.scratch_floats && (rc = S.get(dp.scratch_floats, &s.m_scratch))) return rc;
    } else if (tc) {
        rt = 1;
    } else {
        if (s.jacobi || !plan_sparse_sell(in->dev, R, c->device, &sp))
            sp = plan_sparse(in->dev, R, s.jacobi, c->device);
        // Magnetisations beyond shared memory: every replica resident and each
        // level spread over the whole grid, when all of them fit in half of
        // the free device memory and of what the budget has left (else the
        // per-CTA slabs).
        if (sp.sell && !sp.onchip && env_flag("MARS_SELL_WIDE", 1)) {
            const int wrt = in->dev.shape.sell_rt >= 0 ? in->dev.shape.sell_rt : env_flag("MARS_SELL_RT", 4);
            if (plan_sparse_wide(in->dev, R, wrt, c->device, &wp)) {
                const size_t need = (size_t)wp.groups * wp.slab * sizeof(float);
                size_t free_b = 0, total_b = 0;
                cudaMemGetInfo(&free_b, &total_b);
                wide = 2 * need <= free_b && (!c->budget || c->used + 2 * need <= c->budget);
            }
        }
        if (wide) {
            rt = wp.rt;
        } else {
            rt = sp.rt;
            const size_t per = (size_t)sp.grid * n * rt;
            float* scr = nullptr;
            if (sp.scratch_floats && (rc = S.get(sp.scratch_floats, &scr))) return rc;
            if (!sp.onchip) { s.m_scratch = scr; scr += per; }
            if (s.jacobi) s.m_next = scr;
        }
    }
    std::vector<int32_t> reps(R);
    std::iota(reps.begin(), reps.end(), 0);
    std::stable_sort(reps.begin(), reps.end(), [&](int32_t a, int32_t b) { return t0h[a] > t0h[b]; });
    // Tiles of rt replicas in that order; the sliced-ELL kernel instead treats
    // the list as one queue that its replica slots draw from.
    const int32_t ntiles = (R + rt - 1) / rt;
    std::vector<int32_t> tile_rep((size_t)ntiles * rt, -1);
    for (int32_t q = 0; q < R; ++q) tile_rep[q] = reps[q];
    int32_t* dtile = nullptr;
    if ((rc = S.get(tile_rep.size(), &dtile))) return rc;
    MARS_CUDA(c, cudaMemcpyAsync(dtile, tile_rep.data(), tile_rep.size() * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, st));
    s.tile_rep = dtile;
    s.ntiles = ntiles;
    s.rt = rt;
    TcProfile tcprof;
    LevelProfile lvprof;
    MARS_CUDA(c, cudaEventRecord(c->ev0, st));
    if (tc) {
        const float t0_max = *std::max_element(t0h.begin(), t0h.end());
        if ((rc = run_dense_tc(c, in, p, s, reps, t0_max, S, &tcprof, (p->flags & MARS_POLISH_FP32) != 0)))
            return rc;
    } else if (in->dev.dense) {
        MARS_CUDA(c, launch_dense(in->dev, s, dp, st));
        MARS_CUDA(c, cudaEventRecord(c->ev3, st));
        ++launches;
    } else if (wide) {
        const float t0_max = *std::max_element(t0h.begin(), t0h.end());
        if ((rc = run_sparse_wide(c, in->dev, p, s, wp, t0_max, S, &launches, &lvprof))) return rc;
        MARS_CUDA(c, cudaEventRecord(c->ev3, st));
    } else {
        if (sp.sell)
            MARS_CUDA(c, launch_sparse_sell(in->dev, s, sp, st));
        else
            MARS_CUDA(c, launch_sparse(in->dev, s, sp, st));
        MARS_CUDA(c, cudaEventRecord(c->ev3, st));
        ++launches;
    }
    launches += tcprof.launches;
    if (!in->dev.integer && in->dev.exact_ok) {  // replace the kernels' FP64 sums by exact ones
        MARS_CUDA(c, launch_energy(in->dev, s.sigma, R, s.energy, nullptr, s.status, st));
        ++launches;
    }
    MARS_CUDA(c, cudaEventRecord(c->ev2, st));
    MARS_CUDA(c, launch_best(s, n, in->dev.integer, dbest, dres, st));
    ++launches;
    MARS_CUDA(c, cudaEventRecord(c->ev1, st));
    DevResult hres;
    int32_t hstatus = 0;
    MARS_CUDA(c, cudaMemcpyAsync(&hres, dres, sizeof hres, cudaMemcpyDeviceToHost, st));
    MARS_CUDA(c, cudaMemcpyAsync(&hstatus, s.status, sizeof hstatus, cudaMemcpyDeviceToHost, st));
    if (best_spins)
        MARS_CUDA(c, cudaMemcpyAsync(best_spins, dbest, n, cudaMemcpyDeviceToHost, st));
    if (outs) {
        const cudaMemcpyKind k = odev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (outs->energies) MARS_CUDA(c, cudaMemcpyAsync(outs->energies, s.energy, R * sizeof(double), k, st));
        if (outs->spins) MARS_CUDA(c, cudaMemcpyAsync(outs->spins, s.sigma, (size_t)R * n, k, st));
        if (outs->m_final && !odev)
            MARS_CUDA(c, cudaMemcpyAsync(outs->m_final, s.m_final, (size_t)R * n * sizeof(float), k, st));
        if (outs->t0) MARS_CUDA(c, cudaMemcpyAsync(outs->t0, t0, R * sizeof(float), k, st));
        if (outs->sweeps) MARS_CUDA(c, cudaMemcpyAsync(outs->sweeps, s.sweeps, R * sizeof(int32_t), k, st));
        if (outs->levels) MARS_CUDA(c, cudaMemcpyAsync(outs->levels, s.levels, R * sizeof(int32_t), k, st));
        if (outs->capped) MARS_CUDA(c, cudaMemcpyAsync(outs->capped, s.capped, R * sizeof(int32_t), k, st));
    }
    MARS_CUDA(c, cudaStreamSynchronize(st));
    float ms = 0.f, ms_descent = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    cudaEventElapsedTime(&ms_descent, c->ev0, c->ev3);
    if (hstatus != kDevOk) return fail(c, MARS_EDEVICE, "device status %d", hstatus);
    if (result) {
        std::memset(result, 0, sizeof *result);
        result->best_energy = hres.best_energy;
        result->best_energy_i64 = hres.best_energy_i64;
        result->best_cut = (in->info.total_weight - hres.best_energy) / 2.0;
        result->best_replica = hres.best_replica;
        result->hits = hres.hits;
        result->mean_energy = hres.sum_energy / R;
        result->sweeps = hres.sweeps;
        result->spin_updates = hres.sweeps * (int64_t)n;
        result->levels = hres.levels;
        result->capped_levels = hres.capped;
        result->gpu_seconds = ms * 1e-3;
        result->descent_seconds = ms_descent * 1e-3;
        result->gemm_seconds = tcprof.gemm_seconds;
        result->gemm_launches = tcprof.gemm_launches;
        result->gemm_flops = tcprof.gemm_flops;
        result->kernel_launches = launches;
        result->level_seconds = lvprof.seconds;
        result->level_launches = lvprof.launches;
        result->level_updates = lvprof.updates;
        result->integer = in->dev.integer;
        result->energy_err_bound = (in->dev.integer || in->dev.exact_ok)
                                       ? 0.0
                                       : std::ldexp(in->abs_weight, -53) * (double)(in->info.nnz / 2 + n);
        result->status = MARS_OK;
    }
    return MARS_OK;
}

int mars_solve_batch(mars_ctx* c, int32_t count, const int32_t* insts, const mars_params* params,
                     int8_t* const* best_spins, mars_result* results)
{
    if (!c || count < 1 || !insts || !params) return MARS_EINVAL;
    DeviceGuard g(c->device);
    cudaStream_t st = c->stream;
    Scratch S(c);
    int rc;
    std::vector<Instance*> ins(count);
    std::vector<DevInstance> dins(count);
    std::vector<BatchJob> jobs(count);
    std::vector<DevResult*> dres(count);
    std::vector<int8_t*> dbest(count);
    std::vector<std::vector<float>> t0h_all(count);
    int64_t launches = 0;
    for (int32_t j = 0; j < count; ++j) {
        const mars_params* p = &params[j];
        Instance* in = find(c, insts[j]);
        if (!in) return fail(c, MARS_ENOTFOUND, "unknown instance %d (job %d)", insts[j], j);
        const int32_t R = p->replicas, n = in->dev.n;
        if (in->dev.dense) return fail(c, MARS_EINVAL, "job %d: batched launches take CSR instances", j);
        if (R < 1 || !std::isfinite(p->t_min) || !std::isfinite(p->t_max) || p->t_min > p->t_max ||
            !(p->c_step > 0.0) || !schedule_ok(p) || levels_bound(p, p->t_max) > kMaxLevels ||
            !(p->d_min >= 0.0) ||
            p->k_max < 1 || p->fixed_sweeps < 0)
            return fail(c, MARS_EINVAL, "job %d: bad parameters", j);
        if (p->update != MARS_UPDATE_GS || p->precision != MARS_FP32 || p->method != MARS_METHOD_MARS)
            return fail(c, MARS_EINVAL, "job %d: batched launches run sequential FP32 MARS sweeps", j);
        if ((size_t)R * n > ((size_t)1 << 40)) return fail(c, MARS_EINVAL, "job %d: R*n too large", j);
        ins[j] = in;
        dins[j] = in->dev;
        DevSolve& s = jobs[j].s;
        s.R = R;
        s.seed = p->seed;
        s.stream = p->stream;
        s.c_step = p->c_step;
        s.d_min = (float)p->d_min;
        s.k_max = p->k_max;
        s.fixed_sweeps = p->fixed_sweeps;
        set_schedule(s, p);
        const bool pdev = p->flags & MARS_DEVICE_PTR;
        float* t0 = nullptr;
        if ((rc = S.get(R, &t0))) return rc;
        std::vector<float>& t0h = t0h_all[j];
        t0h.resize(R);
        if (p->t0) {
            MARS_CUDA(c, cudaMemcpyAsync(t0, p->t0, R * sizeof(float),
                                         pdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        } else {
            MARS_CUDA(c, launch_draw(p->seed, p->stream, 0, R, 0, p->t_min, p->t_max, nullptr, t0, st));
            ++launches;
        }
        MARS_CUDA(c, cudaMemcpyAsync(t0h.data(), t0, R * sizeof(float), cudaMemcpyDeviceToHost, st));
        s.t0 = t0;
        if (p->m0) {
            if (pdev) {
                s.m0 = p->m0;
            } else {
                float* m0 = nullptr;
                if ((rc = S.get((size_t)R * n, &m0))) return rc;
                MARS_CUDA(c, cudaMemcpyAsync(m0, p->m0, (size_t)R * n * sizeof(float),
                                             cudaMemcpyHostToDevice, st));
                s.m0 = m0;
            }
        }
        if ((rc = S.get((size_t)R * n, &s.sigma))) return rc;
        if ((rc = S.get(R, &s.energy))) return rc;
        if ((rc = S.get(R, &s.energy_i64))) return rc;
        if ((rc = S.get(R, &s.sweeps))) return rc;
        if ((rc = S.get(R, &s.levels))) return rc;
        if ((rc = S.get(R, &s.capped))) return rc;
        if ((rc = S.get(2, &s.work_counter))) return rc;
        s.status = s.work_counter + 1;
        MARS_CUDA(c, cudaMemsetAsync(s.work_counter, 0, 2 * sizeof(int32_t), st));
        if ((rc = S.get(1, &dres[j]))) return rc;
        if ((rc = S.get(n, &dbest[j]))) return rc;
        jobs[j].in = in->dev;
    }
    // every job's start temperatures, read back once
    MARS_CUDA(c, cudaStreamSynchronize(st));
    for (int32_t j = 0; j < count; ++j) {
        const mars_params* p = &params[j];
        const std::vector<float>& t0h = t0h_all[j];
        DevSolve& s = jobs[j].s;
        const int32_t R = p->replicas;
        for (float v : t0h)
            if (!std::isfinite(v) || levels_bound(p, v) > kMaxLevels)
                return fail(c, MARS_EINVAL, "job %d: start temperatures out of range", j);
        std::vector<int32_t> reps(R);
        std::iota(reps.begin(), reps.end(), 0);
        std::stable_sort(reps.begin(), reps.end(), [&](int32_t a, int32_t b) { return t0h[a] > t0h[b]; });
        int32_t* dq = nullptr;
        if ((rc = S.get(R, &dq))) return rc;
        MARS_CUDA(c, cudaMemcpyAsync(dq, reps.data(), R * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        s.tile_rep = dq;
        s.ntiles = R;
        s.rt = 1;
    }
    BatchPlan bp;
    std::vector<int> fmts(count), rts(count);
    if (!plan_sparse_batch(dins.data(), count, c->device, &bp, fmts.data(), rts.data()))
        return fail(c, MARS_EINVAL, "an instance is too large for the batched on-chip kernel");
    for (int32_t j = 0; j < count; ++j) {
        jobs[j].fmt = fmts[j];
        jobs[j].rt = rts[j];
    }
    BatchJob* djobs = nullptr;
    int32_t* cursor = nullptr;
    if ((rc = S.get(count, &djobs))) return rc;
    if ((rc = S.get(1, &cursor))) return rc;
    MARS_CUDA(c, cudaMemcpyAsync(djobs, jobs.data(), count * sizeof(BatchJob), cudaMemcpyHostToDevice, st));
    MARS_CUDA(c, cudaMemsetAsync(cursor, 0, sizeof(int32_t), st));
    MARS_CUDA(c, cudaEventRecord(c->ev0, st));
    MARS_CUDA(c, launch_sparse_batch(djobs, count, cursor, bp, st));
    MARS_CUDA(c, cudaEventRecord(c->ev2, st));
    ++launches;
    for (int32_t j = 0; j < count; ++j) {
        const DevSolve& s = jobs[j].s;
        if (!dins[j].integer && dins[j].exact_ok) {
            MARS_CUDA(c, launch_energy(dins[j], s.sigma, s.R, s.energy, nullptr, s.status, st));
            ++launches;
        }
        MARS_CUDA(c, launch_best(s, dins[j].n, dins[j].integer, dbest[j], dres[j], st));
        ++launches;
    }
    MARS_CUDA(c, cudaEventRecord(c->ev1, st));
    std::vector<DevResult> hres(count);
    std::vector<int32_t> hstatus(count, 0);
    for (int32_t j = 0; j < count; ++j) {
        MARS_CUDA(c, cudaMemcpyAsync(&hres[j], dres[j], sizeof(DevResult), cudaMemcpyDeviceToHost, st));
        MARS_CUDA(c, cudaMemcpyAsync(&hstatus[j], jobs[j].s.status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        if (best_spins && best_spins[j])
            MARS_CUDA(c, cudaMemcpyAsync(best_spins[j], dbest[j], dins[j].n, cudaMemcpyDeviceToHost, st));
    }
    MARS_CUDA(c, cudaStreamSynchronize(st));
    float ms = 0.f, ms_descent = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    cudaEventElapsedTime(&ms_descent, c->ev0, c->ev2);
    for (int32_t j = 0; j < count; ++j) {
        if (hstatus[j] != kDevOk) return fail(c, MARS_EDEVICE, "job %d: device status %d", j, hstatus[j]);
        if (!results) continue;
        mars_result* r = &results[j];
        std::memset(r, 0, sizeof *r);
        const Instance* in = ins[j];
        r->best_energy = hres[j].best_energy;
        r->best_energy_i64 = hres[j].best_energy_i64;
        r->best_cut = (in->info.total_weight - hres[j].best_energy) / 2.0;
        r->best_replica = hres[j].best_replica;
        r->hits = hres[j].hits;
        r->mean_energy = hres[j].sum_energy / params[j].replicas;
        r->sweeps = hres[j].sweeps;
        r->spin_updates = hres[j].sweeps * (int64_t)dins[j].n;
        r->levels = hres[j].levels;
        r->capped_levels = hres[j].capped;
        r->gpu_seconds = ms * 1e-3;          // the whole batch
        r->descent_seconds = ms_descent * 1e-3;
        r->integer = dins[j].integer;
        r->energy_err_bound = (dins[j].integer || dins[j].exact_ok)
                                  ? 0.0
                                  : std::ldexp(in->abs_weight, -53) * (double)(in->info.nnz / 2 + dins[j].n);
        r->status = MARS_OK;
        r->kernel_launches = launches;  // the whole batch's
    }
    return MARS_OK;
}

int mars_set_shape(mars_ctx* c, int32_t id, const mars_shape* shape)
{
    if (!c) return MARS_EINVAL;
    Instance* in = find(c, id);
    if (!in) return fail(c, MARS_ENOTFOUND, "unknown instance %d", id);
    LaunchShape sh;
    if (shape) {
        auto in_set = [](int32_t v, std::initializer_list<int32_t> allowed) {
            if (v == -1) return true;
            for (int32_t a : allowed)
                if (v == a) return true;
            return false;
        };
        if (!in_set(shape->sell_rt, {1, 2, 4}) || !in_set(shape->sell_threads, {512, 1024}) ||
            !in_set(shape->sell_smem_table, {0, 1}) || !in_set(shape->tc_rpw, {1, 2, 4}) ||
            !in_set(shape->tc_overlap, {0, 1}) || !in_set(shape->tc_pair, {0, 1}))
            return fail(c, MARS_EINVAL, "launch shape value outside its allowed set");
        sh.sell_rt = shape->sell_rt;
        sh.sell_threads = shape->sell_threads;
        sh.sell_smem_table = shape->sell_smem_table;
        sh.tc_rpw = shape->tc_rpw;
        sh.tc_overlap = shape->tc_overlap;
        sh.tc_pair = shape->tc_pair;
    }
    in->dev.shape = sh;
    return MARS_OK;
}

int mars_get_shape(mars_ctx* c, int32_t id, mars_shape* out)
{
    if (!c || !out) return MARS_EINVAL;
    Instance* in = find(c, id);
    if (!in) return fail(c, MARS_ENOTFOUND, "unknown instance %d", id);
    const LaunchShape& sh = in->dev.shape;
    *out = mars_shape{sh.sell_rt, sh.sell_threads, sh.sell_smem_table, sh.tc_rpw, sh.tc_overlap, sh.tc_pair};
    return MARS_OK;
}

int mars_autotune(mars_ctx* c, int32_t id, const mars_params* p, int32_t repeats, mars_shape* best,
                  double* seconds)
{
    if (!c || !p) return MARS_EINVAL;
    Instance* in = find(c, id);
    if (!in) return fail(c, MARS_ENOTFOUND, "unknown instance %d", id);
    if (repeats < 1 || repeats > 100) return fail(c, MARS_EINVAL, "repeats must be in [1, 100]");
    const DevInstance& d = in->dev;
    std::vector<LaunchShape> cands;
    if (d.dense && (p->precision == MARS_BF16 || p->precision == MARS_FP8)) {
        cands.push_back(LaunchShape{});  // the library's plan, following the active replicas
        for (int sched = 0; sched < 3; ++sched)  // plain, overlap, pairs
            for (int rpw : {1, 2, 4}) {
                LaunchShape sh;
                sh.tc_rpw = rpw;
                sh.tc_overlap = sched == 1 ? 1 : 0;
                sh.tc_pair = sched == 2 ? 1 : 0;
                cands.push_back(sh);
            }
    } else if (!d.dense && p->update == MARS_UPDATE_GS && d.slices && (d.sell_pm1 || d.sell_gen)) {
        for (int tab = 1; tab >= (d.sell16 ? 0 : 1); --tab)
            for (int nt : {1024, 512})
                for (int rt : {1, 2, 4}) {
                    LaunchShape sh;
                    sh.sell_rt = rt;
                    sh.sell_threads = nt;
                    sh.sell_smem_table = tab;
                    cands.push_back(sh);
                }
    }
    if (cands.empty()) cands.push_back(d.shape);  // nothing to choose: time the current shape
    const LaunchShape saved = d.shape;
    LaunchShape win = saved;
    double best_t = INFINITY;
    for (const LaunchShape& sh : cands) {
        in->dev.shape = sh;
        double t = INFINITY;
        for (int r = 0; r < repeats; ++r) {
            mars_result res{};
            const int rc = mars_solve(c, id, p, nullptr, nullptr, &res);
            if (rc != MARS_OK) {
                in->dev.shape = saved;
                return rc;
            }
            t = std::min(t, res.descent_seconds);
        }
        if (t < best_t) {
            best_t = t;
            win = sh;
        }
    }
    in->dev.shape = win;
    if (best)
        *best = mars_shape{win.sell_rt, win.sell_threads, win.sell_smem_table, win.tc_rpw, win.tc_overlap, win.tc_pair};
    if (seconds) *seconds = best_t;
    return MARS_OK;
}

int mars_device_check(mars_ctx* c, int32_t budget_us)
{
    if (!c) return MARS_EINVAL;
    if (budget_us < 1 || budget_us > 10000000) return fail(c, MARS_EINVAL, "budget_us must be in [1, 1e7]");
    DeviceGuard g(c->device);
    if (!c->check_flag) {
        MARS_CUDA(c, cudaHostAlloc((void**)&c->check_flag, sizeof(int32_t), cudaHostAllocMapped));
        MARS_CUDA(c, cudaMalloc((void**)&c->check_status, sizeof(int32_t)));
    }
    int32_t* dflag = nullptr;
    MARS_CUDA(c, cudaHostGetDevicePointer((void**)&dflag, c->check_flag, 0));
    *reinterpret_cast<volatile int32_t*>(c->check_flag) = 0;
    MARS_CUDA(c, cudaMemsetAsync(c->check_status, 0, sizeof(int32_t), c->stream));
    int clock_khz = 0;
    cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, c->device);
    if (clock_khz <= 0) clock_khz = 2000000;
    const long long budget_cycles = (long long)budget_us * (clock_khz / 1000);
    MARS_CUDA(c, launch_flag_wait(dflag, budget_cycles, c->check_status, c->stream));
    if (!c->fault_flag) {
        std::atomic_thread_fence(std::memory_order_seq_cst);
        *reinterpret_cast<volatile int32_t*>(c->check_flag) = 1;
    }
    int32_t status = 0;
    MARS_CUDA(c, cudaMemcpyAsync(&status, c->check_status, sizeof status, cudaMemcpyDeviceToHost, c->stream));
    MARS_CUDA(c, cudaStreamSynchronize(c->stream));
    if (status == kDevTimeout) return fail(c, MARS_ETIMEOUT, "the device gave up waiting for the host's flag");
    return status == kDevOk ? MARS_OK : fail(c, MARS_EDEVICE, "device status %d", status);
}

int mars_energy(mars_ctx* c, int32_t id, const int8_t* spins, int32_t count, double* e,
                int64_t* e_i64, uint32_t flags)
{
    if (!c || (!spins && count > 0) || (!e && count > 0) || count < 0) return MARS_EINVAL;
    Instance* in = find(c, id);
    if (!in) return fail(c, MARS_ENOTFOUND, "unknown instance %d", id);
    if (count == 0) return MARS_OK;
    DeviceGuard g(c->device);
    cudaStream_t st = c->stream;
    const bool devp = flags & MARS_DEVICE_PTR;
    const int32_t n = in->dev.n;
    Scratch S(c);
    int rc;
    const int8_t* dsp = spins;
    double* de = e;
    long long* dei = (long long*)e_i64;
    int32_t* dstatus = nullptr;
    if ((rc = S.get(1, &dstatus))) return rc;
    MARS_CUDA(c, cudaMemsetAsync(dstatus, 0, sizeof(int32_t), st));
    if (!devp) {
        int8_t* t = nullptr;
        if ((rc = S.get((size_t)count * n, &t))) return rc;
        MARS_CUDA(c, cudaMemcpyAsync(t, spins, (size_t)count * n, cudaMemcpyHostToDevice, st));
        dsp = t;
        if ((rc = S.get(count, &de))) return rc;
        if (e_i64 && (rc = S.get(count, &dei))) return rc;
    }
    MARS_CUDA(c, launch_energy(in->dev, dsp, count, de, dei, dstatus, st));
    int32_t hstatus = 0;
    MARS_CUDA(c, cudaMemcpyAsync(&hstatus, dstatus, sizeof hstatus, cudaMemcpyDeviceToHost, st));
    if (!devp) {
        MARS_CUDA(c, cudaMemcpyAsync(e, de, count * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (e_i64) MARS_CUDA(c, cudaMemcpyAsync(e_i64, dei, count * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    }
    MARS_CUDA(c, cudaStreamSynchronize(st));
    if (hstatus != kDevOk) return fail(c, MARS_EINVAL, "spins must be +-1");
    return MARS_OK;
}

int mars_draw_replicas(mars_ctx* c, uint64_t seed, uint32_t stream, int32_t r0, int32_t R,
                       int32_t n, double t_min, double t_max, float* m0, float* t0,
                       uint32_t flags)
{
    if (!c || R < 0 || n < 0 || r0 < 0) return MARS_EINVAL;
    if (!std::isfinite(t_min) || !std::isfinite(t_max) || t_min > t_max)
        return fail(c, MARS_EINVAL, "need finite t_min <= t_max");
    if (R == 0) return MARS_OK;
    DeviceGuard g(c->device);
    cudaStream_t st = c->stream;
    const bool devp = flags & MARS_DEVICE_PTR;
    Scratch S(c);
    int rc;
    float* dm = m0;
    float* dt = t0;
    if (!devp) {
        dm = nullptr;
        dt = nullptr;
        if (m0 && (rc = S.get((size_t)R * n, &dm))) return rc;
        if (t0 && (rc = S.get(R, &dt))) return rc;
    }
    MARS_CUDA(c, launch_draw(seed, stream, r0, R, m0 ? n : 0, t_min, t_max, dm, dt, st));
    if (!devp) {
        if (m0) MARS_CUDA(c, cudaMemcpyAsync(m0, dm, (size_t)R * n * sizeof(float), cudaMemcpyDeviceToHost, st));
        if (t0) MARS_CUDA(c, cudaMemcpyAsync(t0, dt, R * sizeof(float), cudaMemcpyDeviceToHost, st));
    }
    MARS_CUDA(c, cudaStreamSynchronize(st));
    return MARS_OK;
}

}  // extern "C"
