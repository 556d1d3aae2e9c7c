// chert_trace_host: the whole hot path of Algorithm 2 on a 2D lattice as one
// call on host buffers -- inputs copied in, cache build (Eq. 4-14, 26),
// lookup and relaxation with parents (Eq. 27-33), raypaths (Eq. 34), the
// traveltime fields and raypaths copied back.  It chains the public entry
// points in caller-provided device scratch and synchronises once at the end.
//
// The sources are relaxed in waves: the first wave's field components fill
// the device's resident CTA slots (two a SM), the rest follow.  Each wave's
// relaxation and raypaths run on the caller's stream, and its results are
// copied back on a copy stream as soon as they are done, so the copies of
// one wave overlap the relaxation of the next.
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace chert {
namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Source node of every (component, field) for the raypaths: field f of
// either component starts at source f / n_modes.
__global__ void field_sources_kernel(const int64_t* __restrict__ src, int nf, int n_modes, int64_t* __restrict__ fsrc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 2 * nf) fsrc[t] = src[(t % nf) / n_modes];
}

// Sources per wave: as many as fill two resident CTAs a SM with their field
// components (2 per field), at least one.
int wave_sources(int n_modes) {
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || n_sm < 1) {
        cudaGetLastError();
        n_sm = 148;
    }
    return std::max(1, (2 * n_sm) / (2 * n_modes));
}

// The copy stream of each device (created once, non-blocking).
cudaStream_t copy_stream() {
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        streams[dev] = nullptr;
    }
    return streams[dev];
}

struct HostLayout {
    size_t classes, cls, src, fsrc, rcv, cache, flag, tauR, tauI, parR, parI, paths, lens, status, ws, total;
    size_t ws_bytes;
    int wave, n_waves;          // sources per wave, waves
};

HostLayout host_layout(int n_classes, int n_modes, int M, int nx, int nz, int n_off, int n_sources, int n_rcv,
                       int64_t cap, int precision) {
    HostLayout L{};
    L.wave = std::min(n_sources, wave_sources(n_modes));
    L.n_waves = (n_sources + L.wave - 1) / L.wave;
    const size_t es = precision == CHERT_FP64 ? 8 : 4;
    const size_t n = (size_t)nx * nz;
    const size_t nf = (size_t)n_sources * n_modes;
    const size_t ne = (size_t)n_modes * n_classes * 4 * M;
    size_t at = 0;
    auto take = [&](size_t bytes) { const size_t p = at; at += align256(bytes); return p; };
    L.classes = take(sizeof(chert_class) * (size_t)n_classes);
    L.cls = take(4 * n);
    L.src = take(8 * (size_t)n_sources);
    L.fsrc = take(8 * 2 * nf);
    L.rcv = take(8 * (size_t)n_rcv);
    L.cache = take(7 * ne * es);             // V, A, Q, rx, rz, theta, vartheta
    L.flag = take(ne);
    L.tauR = take(nf * n * es);
    L.tauI = take(nf * n * es);
    L.parR = take(4 * nf * n);
    L.parI = take(4 * nf * n);
    L.paths = take(8 * 2 * nf * (size_t)n_rcv * (size_t)cap);
    L.lens = take(8 * 2 * nf * (size_t)n_rcv);
    L.status = take(8 * (size_t)L.n_waves);
    L.ws_bytes = chert_traveltime_workspace_bytes_grid(n_modes, n_classes, n_off, precision, L.wave, nx, 1, nz);
    L.ws = take(L.ws_bytes);
    L.total = at;
    return L;
}

}  // namespace
}  // namespace chert

extern "C" size_t chert_trace_host_scratch_bytes(int n_classes, int n_modes, int M, int nx, int nz, int n_off,
                                                 int n_sources, int n_rcv, int64_t path_cap, int precision) {
    if (n_classes < 1 || n_modes < 1 || n_modes > 3 || M < 1 || nx < 1 || nz < 1 || n_off < 1 || n_sources < 1 ||
        n_rcv < 1 || path_cap < 1 || (precision != CHERT_FP64 && precision != CHERT_FP32 && precision != CHERT_MIXED))
        return 0;
    return chert::host_layout(n_classes, n_modes, M, nx, nz, n_off, n_sources, n_rcv, path_cap, precision).total;
}

extern "C" int chert_trace_host(const chert_class* h_classes, int n_classes, const int* modes, int n_modes,
                                const chert_cache_params* params, int nx, int nz, double dx,
                                const int32_t* h_class_of_node, const int32_t* offsets, int n_off,
                                const int64_t* h_sources, int n_sources, int max_cycles, const int64_t* h_receivers,
                                int n_rcv, int64_t path_cap, void* h_tauR, void* h_tauI, int64_t* h_paths,
                                int64_t* h_path_len, void* d_scratch, size_t scratch_bytes, void* stream) {
    using namespace chert;
    const char* who = "chert_trace_host";
    CHERT_REQUIRE(h_classes && modes && params && h_class_of_node && offsets && h_sources && h_receivers &&
                      h_tauR && h_tauI && h_paths && h_path_len && d_scratch,
                  "%s: NULL argument", who);
    const size_t need = chert_trace_host_scratch_bytes(n_classes, n_modes, params->M, nx, nz, n_off, n_sources,
                                                       n_rcv, path_cap, params->precision);
    CHERT_REQUIRE(need > 0, "%s: bad sizes or precision", who);
    if (scratch_bytes < need) {
        set_error("%s: scratch %zu < %zu bytes", who, scratch_bytes, need);
        return CHERT_ENOMEM;
    }
    const int prec = params->precision;
    const HostLayout L = host_layout(n_classes, n_modes, params->M, nx, nz, n_off, n_sources, n_rcv, path_cap, prec);
    unsigned char* d = static_cast<unsigned char*>(d_scratch);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t es = prec == CHERT_FP64 ? 8 : 4;
    const size_t n = (size_t)nx * nz;
    const int nf = n_sources * n_modes;
    const size_t ne = (size_t)n_modes * n_classes * 4 * params->M;

    // inputs in
    cudaError_t e = cudaMemcpyAsync(d + L.classes, h_classes, sizeof(chert_class) * (size_t)n_classes,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d + L.cls, h_class_of_node, 4 * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d + L.src, h_sources, 8 * (size_t)n_sources, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d + L.rcv, h_receivers, 8 * (size_t)n_rcv, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "chert_trace_host: input copies");
    field_sources_kernel<<<(2 * nf + 255) / 256, 256, 0, s>>>(reinterpret_cast<const int64_t*>(d + L.src), nf,
                                                              n_modes, reinterpret_cast<int64_t*>(d + L.fsrc));
    int rc0 = launch_check("chert_trace_host: field sources");
    if (rc0) return rc0;

    chert_cache_arrays cache;
    unsigned char* cb = d + L.cache;
    cache.V = cb;
    cache.A = cb + ne * es;
    cache.Q = cb + 2 * ne * es;
    cache.rx = cb + 3 * ne * es;
    cache.rz = cb + 4 * ne * es;
    cache.theta = cb + 5 * ne * es;
    cache.vartheta = cb + 6 * ne * es;
    cache.flag = d + L.flag;
    cache.ry = nullptr;
    cache.phi = nullptr;
    int rc = chert_build_cache(reinterpret_cast<const chert_class*>(d + L.classes), n_classes, modes, n_modes,
                               params, &cache, s);
    if (rc) return rc;
    int32_t* status = reinterpret_cast<int32_t*>(d + L.status);
    cudaStream_t cs = L.n_waves > 1 ? copy_stream() : nullptr;
    const int waves = cs ? L.n_waves : 1;
    const int wave = cs ? L.wave : n_sources;
    const size_t field_bytes = n * es;
    const size_t path_bytes = 8 * (size_t)n_rcv * path_cap, len_bytes = 8 * (size_t)n_rcv;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    auto cleanup = [&]() {
        for (cudaEvent_t x : ev)
            if (x) cudaEventDestroy(x);
    };
    for (int k = 0; k < 2 && cs; ++k) {
        e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "chert_trace_host: events");
        }
    }
    // the copies of the waves before the last overlap the next wave's work
    auto copy_wave = [&](cudaStream_t cst, int s0, int ns) -> cudaError_t {
        const size_t f0 = (size_t)s0 * n_modes, fn = (size_t)ns * n_modes;
        cudaError_t er = cudaMemcpyAsync(static_cast<unsigned char*>(h_tauR) + f0 * field_bytes,
                                         d + L.tauR + f0 * field_bytes, fn * field_bytes, cudaMemcpyDeviceToHost, cst);
        if (er == cudaSuccess)
            er = cudaMemcpyAsync(static_cast<unsigned char*>(h_tauI) + f0 * field_bytes,
                                 d + L.tauI + f0 * field_bytes, fn * field_bytes, cudaMemcpyDeviceToHost, cst);
        for (int c = 0; c < 2 && er == cudaSuccess; ++c) {
            const size_t g0 = (size_t)c * nf + f0;
            er = cudaMemcpyAsync(reinterpret_cast<unsigned char*>(h_paths) + g0 * path_bytes,
                                 d + L.paths + g0 * path_bytes, fn * path_bytes, cudaMemcpyDeviceToHost, cst);
            if (er == cudaSuccess)
                er = cudaMemcpyAsync(reinterpret_cast<unsigned char*>(h_path_len) + g0 * len_bytes,
                                     d + L.lens + g0 * len_bytes, fn * len_bytes, cudaMemcpyDeviceToHost, cst);
        }
        return er;
    };
    for (int k = 0; k < waves; ++k) {
        const int s0 = k * wave, ns = std::min(wave, n_sources - s0);
        const size_t f0 = (size_t)s0 * n_modes;
        const int nfk = ns * n_modes;
        rc = chert_traveltime_enqueue(&cache, n_modes, n_classes, 4 * params->M, nx, 1, nz, dx,
                                      reinterpret_cast<const int32_t*>(d + L.cls), offsets, n_off,
                                      reinterpret_cast<const int64_t*>(d + L.src) + s0, ns, prec, max_cycles,
                                      d + L.tauR + f0 * field_bytes, d + L.tauI + f0 * field_bytes,
                                      reinterpret_cast<int32_t*>(d + L.parR) + f0 * n,
                                      reinterpret_cast<int32_t*>(d + L.parI) + f0 * n, d + L.ws, L.ws_bytes,
                                      status + 2 * k, s);
        for (int c = 0; c < 2 && !rc; ++c)
            rc = chert_raypath(reinterpret_cast<const int32_t*>(d + (c == 0 ? L.parR : L.parI)) + f0 * n, nfk,
                               (int64_t)n, reinterpret_cast<const int64_t*>(d + L.fsrc) + (size_t)c * nf + f0,
                               reinterpret_cast<const int64_t*>(d + L.rcv), n_rcv, path_cap,
                               reinterpret_cast<int64_t*>(d + L.paths) + ((size_t)c * nf + f0) * n_rcv * path_cap,
                               reinterpret_cast<int64_t*>(d + L.lens) + ((size_t)c * nf + f0) * n_rcv, s);
        if (rc) {
            cleanup();
            return rc;
        }
        if (cs) {
            // this wave's results are done on s: copy them on the copy stream
            e = cudaEventRecord(ev[0], s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[0], 0);
            if (e == cudaSuccess) e = copy_wave(cs, s0, ns);
            if (e != cudaSuccess) {
                cleanup();
                return cuda_fail(e, "chert_trace_host: result copies");
            }
        }
    }

    // results out (the rest), one synchronisation
    std::vector<int32_t> h_status(2 * (size_t)waves, 0);
    const int n_stat = waves;
    if (cs) {
        e = cudaEventRecord(ev[1], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[1], 0);
    } else {
        e = copy_wave(s, 0, n_sources);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_status.data(), status, sizeof(int32_t) * 2 * n_stat, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "chert_trace_host: result copies");
    for (int k = 0; k < n_stat; ++k)
        if (h_status[2 * k + 1]) {
            set_error("%s: class map holds ids outside [0, %d)", who, n_classes);
            return CHERT_EINVAL;
        }
    for (int k = 0; k < n_stat; ++k)
        if (h_status[2 * k] >= 0) {
            const int fc = h_status[2 * k] + 2 * k * wave * n_modes;
            set_error("%s: field %d component %d did not converge in %d cycles", who, fc / 2, fc % 2, max_cycles);
            return CHERT_ETIMEOUT;
        }
    return CHERT_OK;
}
