// C ABI of the GB300 direct inverse NFFT: plan lifecycle, argument checks,
// host/device staging and the per-kernel profiler.  The numerical steps live in
// pattern.cu (index sets), lsq.cu (B_opt), spread.cu and fft.cu (the applies).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>

#include "plan.h"

namespace {

std::atomic<int64_t> g_launches{0};
thread_local std::string g_error;

infft_status fail(infft_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return st;
}

// entry points a plan whose M_sigma is not a power of two (a batch of one problem) lacks
infft_status chirp_only(const char* what) {
    return fail(INFFT_EUNSUPPORTED,
                "%s: a plan whose M_sigma is not a power of two supports set_nodes, precompute, infft_apply, "
                "get_info and copy_plan_data only", what);
}

infft_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? INFFT_ENOMEM : INFFT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool is_device_pointer(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();   // clear the sticky-free error of an unknown host pointer
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void free_plan_buffers(Plan* p) {
    if (p->arena) cudaFree(p->arena);
    p->arena = nullptr;
}

// entries of the objective: one per grid point (overdetermined) or per node (underdetermined)
int64_t objective_count(const Plan* p) { return p->ansatz == INFFT_ANSATZ_UNDERDETERMINED ? p->N : p->Ms; }

infft_status validate_sizes(int64_t M, int64_t N, double sigma, int m, int kernel, double tau, int64_t* Ms_out,
                            int* logMs_out) {
    if (M < 2 || (M & 1)) return fail(INFFT_EINVAL, "M must be even and >= 2 (got %lld)", (long long)M);
    if (N < 1) return fail(INFFT_EINVAL, "N must be >= 1 (got %lld)", (long long)N);
    if (!std::isfinite(sigma) || sigma < 1.0) return fail(INFFT_EINVAL, "sigma must be >= 1 (got %g)", sigma);
    const double msd = sigma * (double)M;
    if (msd > (double)(1 << 30) || msd != std::floor(msd) || ((int64_t)msd & 1))
        return fail(INFFT_EINVAL, "sigma*M must be an even integer (got %.17g)", msd);
    const int64_t Ms = (int64_t)msd;
    if (m < 1 || 2 * (int64_t)m >= Ms)
        return fail(INFFT_EINVAL, "need m >= 1 and 2m < M_sigma (m = %d, M_sigma = %lld)", m, (long long)Ms);
    if (kernel != INFFT_KERNEL_FULL && kernel != INFFT_KERNEL_SYM)
        return fail(INFFT_EINVAL, "kernel must be INFFT_KERNEL_FULL or INFFT_KERNEL_SYM (got %d)", kernel);
    if (!(tau >= 0.0 && tau < 1.0)) return fail(INFFT_EINVAL, "tau must be in [0, 1) (got %g)", tau);
    if ((double)N * (2.0 * m + 1.0) >= 2147483647.0)
        return fail(INFFT_EINVAL, "N (2m+1) must be < 2^31 (N = %lld, m = %d)", (long long)N, m);
    if (Ms > (1 << 24))
        return fail(INFFT_EUNSUPPORTED, "M_sigma = %lld: this build supports M_sigma up to 2^24", (long long)Ms);
    if (Ms & (Ms - 1)) {
        // any even M_sigma = 2M with M <= 8192: the chirp-convolution FFT of the batched form
        if (sigma != 2.0 || M > 8192)
            return fail(INFFT_EUNSUPPORTED,
                        "M_sigma = %lld is not a power of two: supported for sigma = 2 and M <= 8192 only",
                        (long long)Ms);
    }
    int lg = 0;
    while ((int64_t(1) << lg) < Ms) ++lg;
    *Ms_out = Ms;
    *logMs_out = lg;
    return INFFT_OK;
}

template <typename T> infft_status apply_impl(infft_plan_t p, const T* f, T* fhat, infft_stream_t stream) {
    if (!p) return fail(INFFT_EINVAL, "plan is NULL");
    if (!f || !fhat) return fail(INFFT_EINVAL, "f and fhat must not be NULL");
    if (!p->precomputed) return fail(INFFT_ENOTREADY, "infft_apply before infft_precompute");
    if (p->chirp) {
        if (sizeof(T) != 4) return chirp_only("infft_apply_z");
        return infft_batch_apply(p->chirp, (const float*)f, (float*)fhat, stream);
    }
    DeviceGuard g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    const size_t csz = 2 * sizeof(T);
    const void* fin = f;
    cudaError_t e;
    if (!is_device_pointer(f)) {
        if ((e = cudaMemcpyAsync(p->stage_in, f, p->N * csz, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return cuda_fail(e, "copy f to device");
        fin = p->stage_in;
    }
    const bool host_out = !is_device_pointer(fhat);
    void* fout = host_out ? p->stage_out : (void*)fhat;
    if (sizeof(T) == 4 && apply2_default_config(p) >= 0) {
        // two launches: spreading fused with FFT pass A, then pass B with D
        if ((e = run_apply2(p, (const float2*)fin, false, (float2*)fout, s)) != cudaSuccess)
            return cuda_fail(e, "apply");
    } else {
        if ((e = run_spread<T>(p, fin, s)) != cudaSuccess) return cuda_fail(e, "spread");
        if ((e = run_fft_adjoint<T>(p, fout, s)) != cudaSuccess) return cuda_fail(e, "fft");
    }
    if (host_out) {
        if ((e = cudaMemcpyAsync(fhat, p->stage_out, p->M * csz, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_fail(e, "copy fhat to host");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "synchronize");
    }
    return INFFT_OK;
}

template <typename T> infft_status nfft_impl(infft_plan_t p, const T* fhat, T* f, infft_stream_t stream) {
    if (!p) return fail(INFFT_EINVAL, "plan is NULL");
    if (p->chirp) return chirp_only(sizeof(T) == 4 ? "nfft_apply" : "nfft_apply_z");
    if (!f || !fhat) return fail(INFFT_EINVAL, "fhat and f must not be NULL");
    if (!p->precomputed) return fail(INFFT_ENOTREADY, "nfft_apply before infft_precompute");
    DeviceGuard g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    const size_t csz = 2 * sizeof(T);
    const void* in = fhat;
    cudaError_t e;
    if (!is_device_pointer(fhat)) {
        if ((e = cudaMemcpyAsync(p->stage_in, fhat, p->M * csz, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return cuda_fail(e, "copy fhat to device");
        in = p->stage_in;
    }
    const bool host_out = !is_device_pointer(f);
    void* out = host_out ? p->stage_out : (void*)f;
    if ((e = run_fft_forward<T>(p, in, s)) != cudaSuccess) return cuda_fail(e, "fft");
    if ((e = run_interp<T>(p, out, s)) != cudaSuccess) return cuda_fail(e, "interpolate");
    if (host_out) {
        if ((e = cudaMemcpyAsync(f, p->stage_out, p->N * csz, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_fail(e, "copy f to host");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "synchronize");
    }
    return INFFT_OK;
}

}  // namespace

int64_t first_bad_coordinate(const double* x, int64_t n) {
    int64_t bad = 0;
    for (int64_t j = 0; j < n; ++j) bad += !((x[j] >= -0.5) & (x[j] < 0.5));
    if (!bad) return -1;
    for (int64_t j = 0; j < n; ++j)
        if (!(x[j] >= -0.5 && x[j] < 0.5)) return j;
    return -1;
}

infft_status set_error(infft_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return st;
}

void plan_layout(Plan* p, Carver& c, bool member) {
    const int64_t N = p->N, M = p->M, Ms = p->Ms, m = p->m;
    if (!member) c.take(p->x, N);
    c.take(p->xs, N);
    c.take(p->skey, N); c.take(p->perm, N); c.take(p->sort_tmp, N);
    c.take(p->bucket, 2 * Ms + 1); c.take(p->cursor, 2 * Ms); c.take(p->seg_list, N / 32 + 2);
    c.take(p->col_start, Ms); c.take(p->col_count, Ms); c.take(p->col_off, Ms + 1);
    c.take(p->big_list, Ms); c.take(p->list_a, Ms); c.take(p->tiles_mid, Ms / 32 + 2);
    c.take(p->tiles_big, Ms / 32 + 2); c.take(p->tiles_48, Ms / 32 + 2); c.take(p->tiles_64, Ms / 32 + 2);
    c.take(p->scan_sums, (2 * Ms + 1 + 4095) / 4096 + 2);
    c.take(p->phase, N);
    c.take(p->counters, CNT_N);
    c.take(p->w64, p->nnz_cap); c.take(p->w32, p->nnz_cap); c.take(p->J, Ms > N ? Ms : N); c.take(p->wide, Ms);
    c.take(p->wlo, p->nnz_cap);
    if (member) return;
    c.take(p->gterm, p->nnz_cap);
    {
        const int64_t tiles = apply2_max_tiles(p) > 0 ? apply2_max_tiles(p) : 1;
        c.take(p->lay_hdr, tiles);
        c.take(p->lay_cdesc, Ms);
        c.take(p->lay_w, apply2_weight_capacity(p));
        c.take(p->lay_list, apply2_list_capacity(p));
        c.take(p->lay_list_sorted, apply2_list_capacity(p));
        c.take(p->lay_tmp, 5 * tiles);
    }
    if (p->ansatz == INFFT_ANSATZ_UNDERDETERMINED) {
        double2 *ustep, *upart, *umom, *uS;
        c.take(ustep, N); c.take(upart, (int64_t)under_moment_chunks(N) * M); c.take(umom, M);
        c.take(uS, (2 * m + 1) * Ms);
        p->under_step = ustep; p->under_part = upart; p->under_mom = umom; p->under_S = uS;
    }
    const int64_t stage = (N > M ? N : M);
    double2 *grid, *work, *sin_, *sout;
    c.take(grid, Ms); c.take(work, Ms); c.take(sin_, stage); c.take(sout, stage);
    p->grid = grid; p->work = work; p->stage_in = sin_; p->stage_out = sout;
}

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void launch_begin(Plan* p, const char* name, cudaStream_t s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!p->profiling) return;
    ProfileRec r;
    r.name = name;
    cudaEventCreate(&r.start);
    cudaEventCreate(&r.stop);
    cudaEventRecord(r.start, s);
    p->prof.push_back(r);
}

void launch_end(Plan* p, cudaStream_t s) {
    if (!p->profiling || p->prof.empty()) return;
    cudaEventRecord(p->prof.back().stop, s);
}

extern "C" {

infft_status infft_plan_create(int64_t M, int64_t N, double sigma, int m, int kernel, double tau,
                               infft_plan_t* out) {
    return infft_plan_create_ansatz(M, N, sigma, m, kernel, INFFT_ANSATZ_OVERDETERMINED, tau, out);
}

infft_status infft_plan_create_ansatz(int64_t M, int64_t N, double sigma, int m, int kernel, int ansatz,
                                      double tau, infft_plan_t* out) {
    if (!out) return fail(INFFT_EINVAL, "out is NULL");
    *out = nullptr;
    int64_t Ms = 0;
    int logMs = 0;
    infft_status st = validate_sizes(M, N, sigma, m, kernel, tau, &Ms, &logMs);
    if (st != INFFT_OK) return st;
    if (ansatz != INFFT_ANSATZ_OVERDETERMINED && ansatz != INFFT_ANSATZ_UNDERDETERMINED)
        return fail(INFFT_EINVAL, "ansatz must be INFFT_ANSATZ_OVERDETERMINED or INFFT_ANSATZ_UNDERDETERMINED (got %d)",
                    ansatz);
    if (ansatz == INFFT_ANSATZ_UNDERDETERMINED && 2 * m + 1 > UNDER_NMAX)
        return fail(INFFT_EUNSUPPORTED, "underdetermined case: 2m+1 = %d exceeds %d", 2 * m + 1, UNDER_NMAX);
    if (ansatz == INFFT_ANSATZ_UNDERDETERMINED && (Ms & (Ms - 1)))
        return fail(INFFT_EUNSUPPORTED, "the underdetermined case needs M_sigma a power of two");
    int dev = 0, sms = 0;
    cudaError_t qe = cudaGetDevice(&dev);
    if (qe == cudaSuccess) qe = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (qe != cudaSuccess || sms <= 0)
        return fail(INFFT_ECUDA, "cannot query the device's multiprocessor count: %s",
                    qe != cudaSuccess ? cudaGetErrorString(qe) : "count <= 0");
    Plan* p = new Plan();
    p->device = dev;
    p->sms = sms;
    if (Ms & (Ms - 1)) {
        p->M = M; p->N = N; p->Ms = Ms; p->m = m; p->kernel = kernel; p->sigma = sigma; p->tau = tau;
        p->ansatz = ansatz;
        p->logMs = logMs;
        const int64_t Mv = M, Nv = N;
        const infft_status st2 = infft_batch_create(1, &Mv, &Nv, sigma, m, kernel, tau, &p->chirp);
        if (st2 != INFFT_OK) {
            delete p;
            return st2;
        }
        *out = p;
        return INFFT_OK;
    }
    p->M = M; p->N = N; p->Ms = Ms; p->m = m; p->kernel = kernel; p->sigma = sigma; p->tau = tau;
    p->ansatz = ansatz;
    p->logMs = logMs;
    p->nnz_cap = N * (2 * (int64_t)m + 1);
    Carver c;
    plan_layout(p, c, false);
    cudaError_t e = cudaMalloc(&p->arena, c.off);
    if (e == cudaSuccess) {
        c.base = (char*)p->arena;
        c.off = 0;
        plan_layout(p, c, false);
    }
    if (e == cudaSuccess) e = cudaMemset(p->counters, 0, CNT_N * sizeof(int32_t));
    if (e == cudaSuccess) e = phase_table_init();
    if (e != cudaSuccess) {
        free_plan_buffers(p);
        delete p;
        return cuda_fail(e, "allocate plan buffers");
    }
    *out = p;
    return INFFT_OK;
}

infft_status infft_set_nodes(infft_plan_t p, const double* x, infft_stream_t stream) {
    if (!p) return fail(INFFT_EINVAL, "plan is NULL");
    if (!x) return fail(INFFT_EINVAL, "x is NULL");
    if (p->chirp) {
        p->precomputed = 0;
        const infft_status st = infft_batch_set_nodes(p->chirp, x, stream);
        if (st == INFFT_OK) p->nodes_set = 1;
        return st;
    }
    DeviceGuard g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    cudaError_t e;
    if (is_device_pointer(x)) {
        e = cudaMemcpyAsync(p->x, x, p->N * sizeof(double), cudaMemcpyDeviceToDevice, s);
    } else {
        const int64_t j = first_bad_coordinate(x, p->N);
        if (j >= 0) return fail(INFFT_EINVAL, "node x[%lld] = %.17g is not in [-1/2, 1/2)", (long long)j, x[j]);
        e = cudaMemcpyAsync(p->x, x, p->N * sizeof(double), cudaMemcpyHostToDevice, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "copy nodes");
    p->precomputed = 0;
    p->apply_clean = 0;
    p->lay_cfg = -1;
    if ((e = run_pattern(p, s)) != cudaSuccess) return cuda_fail(e, "pattern");
    p->nodes_set = 1;
    return INFFT_OK;
}

infft_status infft_plan(int64_t M, int64_t N, const double* x, double sigma, int m, infft_plan_t* out) {
    infft_status st = infft_plan_create(M, N, sigma, m, INFFT_KERNEL_FULL, 1e-12, out);
    if (st != INFFT_OK) return st;
    st = infft_set_nodes(*out, x, nullptr);
    if (st == INFFT_OK) {
        DeviceGuard g((*out)->device);
        cudaError_t e = cudaStreamSynchronize(nullptr);
        if (e != cudaSuccess) st = cuda_fail(e, "synchronize");
    }
    if (st != INFFT_OK) {
        std::string keep = g_error;
        plan_destroy(*out);
        *out = nullptr;
        g_error = keep;
    }
    return st;
}

infft_status infft_precompute(infft_plan_t p, infft_stream_t stream) {
    if (!p) return fail(INFFT_EINVAL, "plan is NULL");
    if (!p->nodes_set) return fail(INFFT_ENOTREADY, "infft_precompute before infft_set_nodes");
    if (p->chirp) {
        const infft_status st = infft_batch_precompute(p->chirp, stream);
        if (st == INFFT_OK) p->precomputed = 1;
        return st;
    }
    DeviceGuard g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    p->apply_clean = 0;
    p->lay_cfg = -1;
    cudaError_t e = p->ansatz == INFFT_ANSATZ_UNDERDETERMINED ? run_precompute_under(p, s) : run_precompute(p, s);
    if (e != cudaSuccess) return cuda_fail(e, "precompute");
    p->precomputed = 1;
    return INFFT_OK;
}

infft_status infft_apply(infft_plan_t p, const float* f, float* fhat, infft_stream_t stream) {
    return apply_impl<float>(p, f, fhat, stream);
}
infft_status infft_apply_z(infft_plan_t p, const double* f, double* fhat, infft_stream_t stream) {
    return apply_impl<double>(p, f, fhat, stream);
}
infft_status infft_apply_sorted(infft_plan_t p, const float* f, float* fhat, infft_stream_t stream) {
    if (!p) return fail(INFFT_EINVAL, "plan is NULL");
    if (p->chirp) return chirp_only("infft_apply_sorted");
    if (!f || !fhat) return fail(INFFT_EINVAL, "f and fhat must not be NULL");
    if (!p->precomputed) return fail(INFFT_ENOTREADY, "infft_apply_sorted before infft_precompute");
    DeviceGuard g(p->device);
    if (!is_device_pointer(f) || !is_device_pointer(fhat))
        return fail(INFFT_EINVAL, "infft_apply_sorted takes device pointers only");
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    cudaError_t e;
    if (apply2_default_config(p) >= 0) {
        e = run_apply2(p, (const float2*)f, true, (float2*)fhat, s);
    } else {
        // the three-launch path reads through the permutation: undo the sorting into the
        // plan's staging buffer first
        e = run_unsort_values(p, (const float2*)f, (float2*)p->stage_in, s);
        if (e == cudaSuccess) e = run_spread<float>(p, p->stage_in, s);
        if (e == cudaSuccess) e = run_fft_adjoint<float>(p, fhat, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "apply");
    return INFFT_OK;
}

infft_status infft_sort_values(infft_plan_t p, const float* f, float* f_sorted, infft_stream_t stream) {
    if (!p) return fail(INFFT_EINVAL, "plan is NULL");
    if (p->chirp) return chirp_only("infft_sort_values");
    if (!f || !f_sorted || f == f_sorted) return fail(INFFT_EINVAL, "f and f_sorted must be distinct buffers");
    if (!p->nodes_set) return fail(INFFT_ENOTREADY, "infft_sort_values before infft_set_nodes");
    DeviceGuard g(p->device);
    if (!is_device_pointer(f) || !is_device_pointer(f_sorted))
        return fail(INFFT_EINVAL, "infft_sort_values takes device pointers only");
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    cudaError_t e = run_sort_values(p, (const float2*)f, (float2*)f_sorted, s);
    if (e != cudaSuccess) return cuda_fail(e, "sort values");
    return INFFT_OK;
}

int32_t infft_apply_config_count(void) { return apply2_config_count(); }

infft_status infft_apply_config_shape(int32_t id, int32_t* log2_N1, int32_t* columns_per_run) {
    if (id < 0 || id >= apply2_config_count()) return fail(INFFT_EINVAL, "no apply config %d", id);
    apply2_config_shape(id, log2_N1, columns_per_run);
    return INFFT_OK;
}

infft_status infft_set_apply_config(infft_plan_t p, int32_t id) {
    if (!p) return fail(INFFT_EINVAL, "plan is NULL");
    if (p->chirp) return chirp_only("infft_set_apply_config");
    if (id != -1 && !apply2_config_valid(p, id))
        return fail(INFFT_EINVAL, "apply config %d is not valid for M_sigma = %lld", id, (long long)p->Ms);
    p->apply_cfg = id;
    return INFFT_OK;
}

int32_t infft_get_apply_config(infft_plan_t p) {
    if (!p || p->chirp || apply2_default_config(p) < 0) return -1;
    return p->apply_cfg >= 0 ? p->apply_cfg : apply2_default_config(p);
}

infft_status infft_tune_apply(infft_plan_t p, int32_t repeats, float* ms_out, int32_t* best,
                              infft_stream_t stream) {
    if (!p) return fail(INFFT_EINVAL, "plan is NULL");
    if (p->chirp) return chirp_only("infft_tune_apply");
    if (repeats < 1 || repeats > 10000) return fail(INFFT_EINVAL, "repeats must be in [1, 10000] (got %d)", repeats);
    if (!p->precomputed) return fail(INFFT_ENOTREADY, "infft_tune_apply before infft_precompute");
    if (apply2_default_config(p) < 0)
        return fail(INFFT_EUNSUPPORTED, "M_sigma = %lld takes the three-launch apply (no tile shapes)",
                    (long long)p->Ms);
    DeviceGuard g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    const int n = apply2_config_count();
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->stage_in, 0, p->N * sizeof(float2), s);
    const int keep = p->apply_cfg;
    int best_id = -1;
    float best_ms = 0.f;
    for (int id = 0; id < n && e == cudaSuccess; ++id) {
        if (ms_out) ms_out[id] = -1.f;
        if (!apply2_config_valid(p, id)) continue;
        p->apply_cfg = id;
        for (int w = 0; w < 2 && e == cudaSuccess; ++w)
            e = run_apply2(p, (const float2*)p->stage_in, false, (float2*)p->stage_out, s);
        if (e == cudaSuccess) e = cudaEventRecord(a, s);
        for (int r = 0; r < repeats && e == cudaSuccess; ++r)
            e = run_apply2(p, (const float2*)p->stage_in, false, (float2*)p->stage_out, s);
        if (e == cudaSuccess) e = cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        ms /= (float)repeats;
        if (ms_out) ms_out[id] = ms;
        if (e == cudaSuccess && (best_id < 0 || ms < best_ms)) {
            best_id = id;
            best_ms = ms;
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) {
        p->apply_cfg = keep;
        return cuda_fail(e, "tune apply");
    }
    p->apply_cfg = best_id;
    if (best) *best = best_id;
    return INFFT_OK;
}

int64_t infft_apply_many_workspace(infft_plan_t p, int64_t K) {
    if (!p || p->chirp || K < 1) return 0;
    return 2 * K * p->Ms * (int64_t)sizeof(float2) + 256;
}

infft_status infft_apply_many(infft_plan_t p, int64_t K, const float* f, float* fhat, void* workspace,
                              int64_t workspace_bytes, infft_stream_t stream) {
    if (!p) return fail(INFFT_EINVAL, "plan is NULL");
    if (p->chirp) return chirp_only("infft_apply_many");
    if (!f || !fhat || !workspace) return fail(INFFT_EINVAL, "f, fhat and workspace must not be NULL");
    if (K < 1 || K > 65535) return fail(INFFT_EINVAL, "K must be in [1, 65535] (got %lld)", (long long)K);
    if (!p->precomputed) return fail(INFFT_ENOTREADY, "infft_apply_many before infft_precompute");
    if (p->Ms <= 2048) return fail(INFFT_EUNSUPPORTED, "infft_apply_many needs M_sigma > 2048 (got %lld)",
                                   (long long)p->Ms);
    if (workspace_bytes < infft_apply_many_workspace(p, K))
        return fail(INFFT_EINVAL, "workspace of %lld bytes is smaller than infft_apply_many_workspace() = %lld",
                    (long long)workspace_bytes, (long long)infft_apply_many_workspace(p, K));
    DeviceGuard g(p->device);
    if (!is_device_pointer(f) || !is_device_pointer(fhat) || !is_device_pointer(workspace))
        return fail(INFFT_EINVAL, "infft_apply_many takes device pointers only");
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    char* ws = (char*)(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    void* grid = ws;
    void* work = ws + K * p->Ms * sizeof(float2);
    cudaError_t e;
    // the spreading stages each tile's weights and node indices once for all K vectors (faster
    // here than the fused apply's kernels with one CTA row per vector: 76 against 117 us at K = 16)
    if ((e = run_spread_many(p, f, grid, (int)K, s)) != cudaSuccess) return cuda_fail(e, "spread");
    if ((e = run_fft_adjoint_many(p, grid, work, fhat, (int)K, s)) != cudaSuccess) return cuda_fail(e, "fft");
    return INFFT_OK;
}

infft_status infft_ndft_z(infft_plan_t p, const double* fhat, double* f, infft_stream_t stream) {
    if (!p) return fail(INFFT_EINVAL, "plan is NULL");
    if (p->chirp) return chirp_only("infft_ndft_z");
    if (!fhat || !f) return fail(INFFT_EINVAL, "fhat and f must not be NULL");
    if (!p->nodes_set) return fail(INFFT_ENOTREADY, "infft_ndft_z before infft_set_nodes");
    DeviceGuard g(p->device);
    if (!is_device_pointer(fhat) || !is_device_pointer(f))
        return fail(INFFT_EINVAL, "infft_ndft_z takes device pointers only");
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    cudaError_t e = run_ndft_z(p, fhat, nullptr, f, s);
    if (e != cudaSuccess) return cuda_fail(e, "direct sum");
    return INFFT_OK;
}

infft_status infft_nfft_kb_z(infft_plan_t p, const double* fhat, double* f, infft_stream_t stream) {
    if (!p) return fail(INFFT_EINVAL, "plan is NULL");
    if (p->chirp) return chirp_only("infft_nfft_kb_z");
    if (!fhat || !f) return fail(INFFT_EINVAL, "fhat and f must not be NULL");
    if (!p->nodes_set) return fail(INFFT_ENOTREADY, "infft_nfft_kb_z before infft_set_nodes");
    if (!nfft_kb_supported(p))
        return fail(INFFT_EUNSUPPORTED, "infft_nfft_kb_z needs sigma >= 2 and M_sigma >= 96 (M_sigma = %lld)",
                    (long long)p->Ms);
    DeviceGuard g(p->device);
    if (!is_device_pointer(fhat) || !is_device_pointer(f))
        return fail(INFFT_EINVAL, "infft_nfft_kb_z takes device pointers only");
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    cudaError_t e = run_nfft_kb_z(p, fhat, nullptr, f, p->stage_out, s);
    if (e != cudaSuccess) return cuda_fail(e, "windowed NFFT");
    return INFFT_OK;
}

infft_status infft_refine_z(infft_plan_t p, const double* f, double* fhat, int sweeps, infft_stream_t stream) {
    if (!p) return fail(INFFT_EINVAL, "plan is NULL");
    if (p->chirp) return chirp_only("infft_refine_z");
    if (!f || !fhat) return fail(INFFT_EINVAL, "f and fhat must not be NULL");
    if (sweeps < 0 || sweeps > 64) return fail(INFFT_EINVAL, "sweeps must be in [0, 64] (got %d)", sweeps);
    if (!p->precomputed) return fail(INFFT_ENOTREADY, "infft_refine_z before infft_precompute");
    DeviceGuard g(p->device);
    if (!is_device_pointer(f) || !is_device_pointer(fhat))
        return fail(INFFT_EINVAL, "infft_refine_z takes device pointers only");
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    double* r = (double*)p->stage_in;       // N complex128: the residual f - A fhat
    double* d = (double*)p->stage_out;      // M complex128: its inverse NFFT
    const bool fast = nfft_kb_supported(p);
    for (int it = 0; it < sweeps; ++it) {
        cudaError_t e = fast ? run_nfft_kb_z(p, fhat, f, r, d, s) : run_ndft_z(p, fhat, f, r, s);
        if (e != cudaSuccess) return cuda_fail(e, "residual");
        const infft_status st = apply_impl<double>(p, r, d, stream);
        if (st != INFFT_OK) return st;
        if ((e = run_axpy_z(p, fhat, d, (int)p->M, s)) != cudaSuccess) return cuda_fail(e, "update");
    }
    return INFFT_OK;
}

infft_status nfft_apply(infft_plan_t p, const float* fhat, float* f, infft_stream_t stream) {
    return nfft_impl<float>(p, fhat, f, stream);
}
infft_status nfft_apply_z(infft_plan_t p, const double* fhat, double* f, infft_stream_t stream) {
    return nfft_impl<double>(p, fhat, f, stream);
}

infft_status infft_grad_nodes(infft_plan_t p, const float* f, const float* w, double* grad_x,
                              infft_stream_t stream) {
    if (!p) return fail(INFFT_EINVAL, "plan is NULL");
    if (p->chirp) return chirp_only("infft_grad_nodes");
    if (!f || !w || !grad_x) return fail(INFFT_EINVAL, "f, w and grad_x must not be NULL");
    if (!p->precomputed) return fail(INFFT_ENOTREADY, "infft_grad_nodes before infft_precompute");
    if (p->ansatz != INFFT_ANSATZ_OVERDETERMINED)
        return fail(INFFT_EUNSUPPORTED, "infft_grad_nodes: underdetermined plans have no node gradient");
    DeviceGuard g(p->device);
    if (!is_device_pointer(f) || !is_device_pointer(w) || !is_device_pointer(grad_x))
        return fail(INFFT_EINVAL, "infft_grad_nodes takes device pointers only");
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    cudaError_t e = run_grad_nodes(p, f, w, grad_x, s);
    if (e != cudaSuccess) return cuda_fail(e, "node gradient");
    return INFFT_OK;
}

infft_status plan_destroy(infft_plan_t p) {
    if (!p) return INFFT_OK;
    if (p->chirp) {
        const infft_status st = infft_batch_destroy(p->chirp);
        delete p;
        return st;
    }
    {
        DeviceGuard g(p->device);
        cudaDeviceSynchronize();
        for (auto& r : p->prof) { cudaEventDestroy(r.start); cudaEventDestroy(r.stop); }
        free_plan_buffers(p);
    }
    delete p;
    return INFFT_OK;
}

infft_status infft_get_info(infft_plan_t p, infft_info* info) {
    if (!p || !info) return fail(INFFT_EINVAL, "plan and info must not be NULL");
    if (p->chirp) {
        infft_batch_info bi;
        const infft_status st = infft_batch_get_info(p->chirp, &bi);
        if (st != INFFT_OK) return st;
        std::memset(info, 0, sizeof *info);
        info->M = p->M; info->N = p->N; info->M_sigma = p->Ms; info->m = p->m; info->kernel = p->kernel;
        info->sigma = p->sigma; info->tau = p->tau; info->ansatz = p->ansatz;
        info->nodes_set = p->nodes_set; info->precomputed = p->precomputed;
        info->nnz = bi.nnz; info->max_column = bi.max_column; info->empty_columns = (int32_t)bi.empty_columns;
        info->bad_nodes = (int32_t)bi.bad_nodes; info->fallback_columns = (int32_t)bi.fallback_columns;
        info->unsupported_columns = (int32_t)bi.unsupported_columns; info->objective = bi.objective;
        return INFFT_OK;
    }
    DeviceGuard g(p->device);
    cudaError_t e = cudaStreamSynchronize(p->last_stream);
    if (e != cudaSuccess) return cuda_fail(e, "synchronize");
    int32_t cnt[CNT_N];
    if ((e = cudaMemcpy(cnt, p->counters, sizeof cnt, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "read counters");
    std::memset(info, 0, sizeof *info);
    info->M = p->M; info->N = p->N; info->M_sigma = p->Ms; info->m = p->m; info->kernel = p->kernel;
    info->sigma = p->sigma; info->tau = p->tau;
    info->ansatz = p->ansatz;
    info->nodes_set = p->nodes_set;
    info->precomputed = p->precomputed;
    if (p->nodes_set) {
        int32_t nnz = 0;
        if ((e = cudaMemcpy(&nnz, p->col_off + p->Ms, sizeof nnz, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(e, "read nnz");
        info->nnz = nnz;
        info->max_column = cnt[CNT_MAX_COLUMN];
        info->empty_columns = cnt[CNT_EMPTY];
        info->bad_nodes = cnt[CNT_BAD_NODES];
    }
    if (p->precomputed) {
        info->fallback_columns = cnt[CNT_FALLBACK];
        info->unsupported_columns = cnt[CNT_UNSUPPORTED];
        info->grad_failed_columns = cnt[CNT_GRAD_FAIL];
        const int64_t nJ = objective_count(p);
        std::string buf(nJ * sizeof(double), '\0');
        if ((e = cudaMemcpy(&buf[0], p->J, nJ * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(e, "read objective");
        const double* J = (const double*)buf.data();
        double sum = 0.0;
        for (int64_t i = 0; i < nJ; ++i) sum += J[i];
        info->objective = sum;
    }
    return INFFT_OK;
}

infft_status infft_copy_plan_data(infft_plan_t p, int32_t* perm, int32_t* col_start, int32_t* col_count,
                                  int32_t* col_offset, double* weights, double* objective) {
    if (!p) return fail(INFFT_EINVAL, "plan is NULL");
    if (p->chirp) return infft_batch_copy_problem(p->chirp, 0, perm, col_start, col_count, col_offset, weights, objective);
    if (!p->nodes_set) return fail(INFFT_ENOTREADY, "no nodes set");
    if ((weights || objective) && !p->precomputed) return fail(INFFT_ENOTREADY, "not precomputed");
    DeviceGuard g(p->device);
    cudaError_t e = cudaStreamSynchronize(p->last_stream);
    if (e != cudaSuccess) return cuda_fail(e, "synchronize");
    int32_t nnz = 0;
    e = cudaMemcpy(&nnz, p->col_off + p->Ms, sizeof nnz, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && perm) e = cudaMemcpy(perm, p->perm, p->N * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && col_start) e = cudaMemcpy(col_start, p->col_start, p->Ms * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && col_count) e = cudaMemcpy(col_count, p->col_count, p->Ms * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && col_offset) e = cudaMemcpy(col_offset, p->col_off, (p->Ms + 1) * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && weights) e = cudaMemcpy(weights, p->w64, (size_t)nnz * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && objective) e = cudaMemcpy(objective, p->J, objective_count(p) * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "copy plan data");
    return INFFT_OK;
}

infft_status infft_profile(infft_plan_t p, int enable) {
    if (!p) return fail(INFFT_EINVAL, "plan is NULL");
    p->profiling = enable != 0;
    return INFFT_OK;
}

infft_status infft_profile_read(infft_plan_t p, int cap, const char** names, int64_t* launches,
                                double* milliseconds, int* n) {
    if (!p || !n) return fail(INFFT_EINVAL, "plan and n must not be NULL");
    DeviceGuard g(p->device);
    std::map<std::string, std::pair<int64_t, double>> agg;
    std::map<std::string, const char*> keep;
    for (auto& r : p->prof) {
        cudaEventSynchronize(r.stop);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.start, r.stop);
        auto& a = agg[r.name];
        a.first += 1;
        a.second += ms;
        keep[r.name] = r.name;
        cudaEventDestroy(r.start);
        cudaEventDestroy(r.stop);
    }
    p->prof.clear();
    int i = 0;
    for (auto& kv : agg) {
        if (i >= cap) break;
        if (names) names[i] = keep[kv.first];
        if (launches) launches[i] = kv.second.first;
        if (milliseconds) milliseconds[i] = kv.second.second;
        ++i;
    }
    *n = i;
    return INFFT_OK;
}

int64_t infft_launch_count(void) { return g_launches.load(); }

const char* infft_last_error(void) { return g_error.c_str(); }

const char* infft_version(void) { return "infft-gb300 0.1 (sm_103a)"; }

}  // extern "C"
