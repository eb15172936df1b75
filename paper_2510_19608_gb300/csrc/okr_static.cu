// okr_static.cu -- okr_power_flow_static: the load flow of okr_power_flow for
// callers that must not allocate device memory.  Its scratch memory is one
// file-scope __device__ array; nothing here calls cudaMalloc, cudaFree or an
// allocating library routine.
//
// Who needs this: code embedded in a host framework whose allocator owns the
// device memory (a cudaMalloc there fails, or escapes the framework's
// accounting), and loops that cannot take the implicit device-wide
// synchronisation of cudaMalloc/cudaFree.  Such callers bring their own input
// and output buffers; this file supplies the rest from the static array.
//
// The array's name is a host-side stand-in in host code, not a device
// address: its device address is fetched with cudaGetSymbolAddress once per
// device, on the first call made with that device current, and passed to the
// kernels from then on.
#include "okron.h"
#include "okr_internal.cuh"
#include "okr_kernels.cuh"

#include <mutex>

using namespace okr;

namespace {

constexpr int kStaticMaxBus = OKR_STATIC_MAX_BUS;
constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;

constexpr size_t round_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

// Bytes of scratch for a feeder of n buses and L scenarios, in the order
// carve() lays them out (each piece starts on a 256-byte boundary).
constexpr size_t scratch_bytes(size_t n, size_t L) {
    return round_up(sizeof(int) * n) * 5                    // dep, anc, anc2, d2, size
         + round_up(sizeof(int) * (n + 2))                  // ccount
         + round_up(sizeof(int) * (n + 1))                  // coff_c
         + round_up(sizeof(int) * n)                        // child_c
         + round_up(sizeof(int) * 2)                        // T.maxd
         + round_up(sizeof(int) * n) * 5                    // T.parent, orig, pre, sz, depth
         + round_up(sizeof(int) * (n + 1))                  // T.child_off
         + round_up(sizeof(int) * n)                        // T.child
         + round_up(sizeof(int) * (n + 2))                  // T.level_off
         + round_up(sizeof(int) * n)                        // T.level_bus
         + round_up(n)                                      // T.ph
         + round_up(sizeof(double2) * 9 * n) * 3            // T.zl, yl, zc
         + round_up(sizeof(float2) * 9 * n) * 2             // T.zh, zlo
         + round_up(sizeof(double2) * 3 * L * n) * 3        // T.vhat, T.ihat, line currents J
         + round_up(sizeof(double) * 3 * L * n)             // T.amag
         + round_up(sizeof(double2) * 3)                    // T.vslack
         + round_up(sizeof(int) * L)                        // sweeps per scenario
         + round_up(sizeof(int));                           // error flag
}

constexpr size_t kScratchBytes = scratch_bytes(kStaticMaxBus, kMaxScen);
static_assert(kScratchBytes == 5396480, "okron.h states the size of the static scratch");

// The scratch: every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceSlot {
    bool ready = false;
    unsigned char *base = nullptr;    // device address of g_scratch on this device
    int num_sms = 0;
};

std::mutex g_setup_mutex;
DeviceSlot g_slots[kMaxDevices];

// Once per device, with that device current: the device address of the scratch.
okr_status device_setup(int dev, DeviceSlot *out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSlot &s = g_slots[dev];
    if (!s.ready) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) return OKR_ECUDA;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            return OKR_ECUDA;
        s.base = static_cast<unsigned char *>(ptr);
        s.num_sms = sms;
        s.ready = true;
    }
    *out = s;
    return OKR_OK;
}

struct Carve {
    unsigned char *p;
    template <typename T>
    T *take(size_t count) {
        T *q = reinterpret_cast<T *>(p);
        p += round_up(sizeof(T) * count);
        return q;
    }
};

struct Scratch {
    int *dep, *anc, *anc2, *d2, *size, *ccount, *coff_c, *child_c;
    double2 *J;
    int *sweeps, *err;
    Topo T;
};

// Same order and sizes as scratch_bytes().
Scratch carve(unsigned char *base, int n, int L) {
    Carve c{base};
    Scratch s{};
    const size_t N = n, NL3 = (size_t)3 * L * n;
    s.dep = c.take<int>(N);
    s.anc = c.take<int>(N);
    s.anc2 = c.take<int>(N);
    s.d2 = c.take<int>(N);
    s.size = c.take<int>(N);
    s.ccount = c.take<int>(N + 2);
    s.coff_c = c.take<int>(N + 1);
    s.child_c = c.take<int>(N);
    Topo &T = s.T;
    T.n = n;
    T.L = L;
    T.maxd = c.take<int>(2);
    T.parent = c.take<int>(N);
    T.orig = c.take<int>(N);
    T.pre = c.take<int>(N);
    T.sz = c.take<int>(N);
    T.depth = c.take<int>(N);
    T.child_off = c.take<int>(N + 1);
    T.child = c.take<int>(N);
    T.level_off = c.take<int>(N + 2);
    T.level_bus = c.take<int>(N);
    T.ph = c.take<uint8_t>(N);
    T.zl = c.take<double2>(9 * N);
    T.yl = c.take<double2>(9 * N);
    T.zc = c.take<double2>(9 * N);
    T.zh = c.take<float2>(9 * N);
    T.zlo = c.take<float2>(9 * N);
    T.vhat = c.take<double2>(NL3);
    T.ihat = c.take<double2>(NL3);
    s.J = c.take<double2>(NL3);
    T.amag = c.take<double>(NL3);
    T.vslack = c.take<double2>(3);
    s.sweeps = c.take<int>((size_t)L);
    s.err = c.take<int>(1);
    T.lca = nullptr;                  // the load flow needs no LCA table
    return s;
}

// Preorder-numbered Vhat / Ihat -> caller layout [L][n][3][2], 0 on absent phases.
__global__ void k_export_static(Topo T, double *vhat_out, double *ihat_out) {
    const int n = T.n, L = T.L;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L * n; e += gridDim.x * blockDim.x) {
        const int l = e / n, i = e % n;
        const int v = T.pre[i];
        for (int p = 0; p < 3; ++p) {
            const bool on = T.ph[v] >> p & 1u;
            const size_t o = (((size_t)l * n + i) * 3 + p) * 2;
            const double2 vh = on ? T.vhat[sidx(l, p, v, n)] : make_double2(0.0, 0.0);
            vhat_out[o] = vh.x;
            vhat_out[o + 1] = vh.y;
            if (ihat_out) {
                const double2 ih = on ? T.ihat[sidx(l, p, v, n)] : make_double2(0.0, 0.0);
                ihat_out[o] = ih.x;
                ihat_out[o + 1] = ih.y;
            }
        }
    }
}

int grid_for(size_t work, int num_sms) {
    size_t b = (work + 255) / 256;
    if (b < 1) b = 1;
    if (b > (size_t)num_sms * 8) b = (size_t)num_sms * 8;
    return (int)b;
}

okr_status read_err(const int *err_dev, cudaStream_t st) {
    int e = 0;
    if (cudaMemcpyAsync(&e, err_dev, sizeof e, cudaMemcpyDeviceToHost, st) != cudaSuccess) return OKR_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return OKR_ECUDA;
    if (e == 1) return OKR_EINVAL;
    if (e == 2) return OKR_ESINGULAR;
    if (e == 3) return OKR_EPF;
    if (e == 6) return OKR_ETIMEOUT;
    return e ? OKR_EINTERNAL : OKR_OK;
}

constexpr double kPfTol = 1e-13;
constexpr int kPfMaxIter = 200;
constexpr long long kPfSpins = 1000000;     // polls per grid barrier of the load flow: under a second

}  // namespace

extern "C" okr_status okr_power_flow_static(const okr_feeder *f, double *vhat_out, double *ihat_out,
                                            int32_t *sweeps, void *stream) {
    if (!f || !vhat_out) return OKR_EINVAL;
    if (f->n_bus < 2 || f->n_bus > kStaticMaxBus) return OKR_EINVAL;
    if (f->n_scen < 1 || f->n_scen > kMaxScen) return OKR_EINVAL;
    if (!f->parent || !f->phases || !f->z_line || !f->s_load) return OKR_EINVAL;
    const int n = f->n_bus, L = f->n_scen;
    if (scratch_bytes(n, L) > kScratchBytes) return OKR_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return OKR_ECUDA;
    if (dev >= kMaxDevices) return OKR_EINVAL;
    DeviceSlot slot;
    okr_status s = device_setup(dev, &slot);
    if (s != OKR_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Scratch w = carve(slot.base, n, L);
    Topo &T = w.T;

    // what must start at zero: the error flag (everything else is written
    // before it is read by the kernels below)
    if (cudaMemsetAsync(w.err, 0, sizeof(int), st) != cudaSuccess) return OKR_ECUDA;
    double2 vs[3];
    for (int p = 0; p < 3; ++p) vs[p] = make_double2(f->v_slack[p][0], f->v_slack[p][1]);
    if (cudaMemcpyAsync(T.vslack, vs, sizeof vs, cudaMemcpyHostToDevice, st) != cudaSuccess) return OKR_ECUDA;

    k_topology<<<1, 1024, 0, st>>>(n, f->parent, f->phases, T, w.dep, w.anc, w.anc2, w.d2, w.size, w.ccount,
                                   w.coff_c, w.child_c, w.err);
    if (cudaGetLastError() != cudaSuccess) return OKR_ECUDA;
    // the next kernels index with the renumbering: stop on an invalid tree
    s = read_err(w.err, st);
    if (s != OKR_OK) return s;
    k_child_offsets<<<1, 1024, 0, st>>>(n, T, w.coff_c, w.child_c);
    if (launch_lines(n, T, f->z_line, w.err, slot.num_sms, st) != cudaSuccess) return OKR_ECUDA;
    // a singular line block (err = 2) stops here, as okr_power_flow does: the
    // load flow would run on undefined admittances and its own outcome would
    // overwrite the flag
    s = read_err(w.err, st);
    if (s != OKR_OK) return s;
    // the load flow's work buffers alias T.ihat and T.amag, which the next two kernels fill
    if (launch_power_flow(n, L, T, f->s_load, kPfTol, kPfMaxIter, w.J, T.ihat, T.amag, w.sweeps, w.err,
                          slot.num_sms, st, kPfSpins) != cudaSuccess)
        return OKR_ECUDA;
    k_line_currents<<<grid_for((size_t)L * n, slot.num_sms), 256, 0, st>>>(n, L, T, w.J);
    k_injections<<<grid_for((size_t)L * n, slot.num_sms), 256, 0, st>>>(n, L, T, w.J);
    k_export_static<<<grid_for((size_t)L * n, slot.num_sms), 256, 0, st>>>(T, vhat_out, ihat_out);
    if (cudaGetLastError() != cudaSuccess) return OKR_ECUDA;
    s = read_err(w.err, st);
    if (s != OKR_OK) return s;
    if (sweeps) {
        int it[kMaxScen];
        if (cudaMemcpyAsync(it, w.sweeps, sizeof(int) * L, cudaMemcpyDeviceToHost, st) != cudaSuccess) return OKR_ECUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return OKR_ECUDA;
        int m = 0;
        for (int l = 0; l < L; ++l) m = it[l] > m ? it[l] : m;
        *sweeps = m;
    }
    return OKR_OK;
}
