// vi_noalloc.cu -- vi_energy_noalloc: the energy reduction (Eq. 1) for callers
// that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc: a serving process whose
// device memory is entirely handed out by its own allocator under a fixed
// memory budget (an unplanned allocation could exceed the budget or fragment
// the pool), or a latency-bound loop sharing the GPU with other work, where
// the device-wide synchronisation that cudaMalloc / cudaFree can imply is not
// acceptable. This entry point reads caller-owned buffers, writes a
// caller-owned output, and keeps its only scratch -- one pair of partial sums
// per thread block -- in a fixed array in the library's static device memory.
//
// The scratch array is `g_energy_scratch` below: VI_NOALLOC_MAX_BLOCKS blocks
// of 256 voxels, i.e. at most VI_NOALLOC_MAX_VOXELS voxels per call; every GPU
// that loads the library holds its 1 MiB until the process exits. Every call
// shares the array, and a call reads back only the slots it has just written,
// so nothing needs clearing between calls; two calls that overlap on the GPU
// (on different streams, or from different threads) race on it.
#include <cuda.h>

#include <mutex>

#include "vi.h"
#include "vi_launch.h"

namespace vi {

static constexpr int NOALLOC_BLOCK = 256;
static constexpr int VI_NOALLOC_MAX_BLOCKS = 65536;
static constexpr long long VI_NOALLOC_MAX_VOXELS = (long long)VI_NOALLOC_MAX_BLOCKS * NOALLOC_BLOCK;

// Per-block (E_H, E_H~) partial sums of the last call.
static __device__ __align__(256) double g_energy_scratch[2 * VI_NOALLOC_MAX_BLOCKS];

// Squared patch distance on the [V][C] layout of the ABI (Eq. 2 / Eq. 7b), in
// the library's summation order: per row (fixed dt, dy) fused multiply-adds
// over dx and channels from 0, row sums added in dy order, slice sums in dt
// order, divided by N = 125.
__device__ float d2_abi_layout(const float *__restrict__ x, int C, int W, int H, int T, int px, int py,
                               int pt, int sx, int sy, int st)
{
    float total = 0.0f;
    for (int dt = -2; dt <= 2; ++dt) {
        const int rt = pt + dt;
        float slice = 0.0f;
        for (int dy = -2; dy <= 2; ++dy) {
            const int ry = py + dy;
            float row = 0.0f;
            if ((unsigned)rt < (unsigned)T && (unsigned)ry < (unsigned)H) {
                for (int dx = -2; dx <= 2; ++dx) {
                    const int rx = px + dx;
                    if ((unsigned)rx >= (unsigned)W)
                        continue;
                    const long long r = ((long long)rt * H + ry) * W + rx;
                    const long long s = ((long long)(st + dt) * H + (sy + dy)) * W + (sx + dx);
                    for (int c = 0; c < C; ++c) {
                        const float df = __fsub_rn(x[r * C + c], x[s * C + c]);
                        row = __fmaf_rn(df, df, row);
                    }
                }
            }
            slice = __fadd_rn(slice, row);
        }
        total = __fadd_rn(total, slice);
    }
    return __fdiv_rn(total, 125.0f);
}

// One thread per voxel; targets (code bit 1) add d^2(W_p, W_{p+phi(p)}) to
// E_H~, and occluded targets (bit 0) to E_H; block sums go to the scratch.
__global__ void __launch_bounds__(NOALLOC_BLOCK)
k_energy_noalloc(const float *__restrict__ x, int C, const int32_t *__restrict__ phi,
                 const uint8_t *__restrict__ code, int W, int H, int T, double *__restrict__ scratch)
{
    __shared__ double sh[2][NOALLOC_BLOCK];
    const long long V = (long long)W * H * T;
    const long long v = (long long)blockIdx.x * NOALLOC_BLOCK + threadIdx.x;
    double eh = 0.0, et = 0.0;
    if (v < V && (code[v] & CODE_TARGET)) {
        const int px = (int)(v % W), py = (int)((v / W) % H), pt = (int)(v / ((long long)W * H));
        const int sx = px + phi[3 * v], sy = py + phi[3 * v + 1], st = pt + phi[3 * v + 2];
        double d = __longlong_as_double(0x7ff0000000000000ll);
        if (sx >= 2 && sx < W - 2 && sy >= 2 && sy < H - 2 && st >= 2 && st < T - 2)
            d = (double)d2_abi_layout(x, C, W, H, T, px, py, pt, sx, sy, st);
        et = d;
        if (code[v] & CODE_HOLE)
            eh = d;
    }
    sh[0][threadIdx.x] = eh;
    sh[1][threadIdx.x] = et;
    __syncthreads();
    for (int o = NOALLOC_BLOCK / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scratch[2 * blockIdx.x] = sh[0][0];
        scratch[2 * blockIdx.x + 1] = sh[1][0];
    }
}

// Sums the n_blocks partial pairs in a fixed order into out[0..1].
__global__ void k_energy_noalloc_sum(const double *__restrict__ scratch, int n_blocks, double *out)
{
    __shared__ double s[2][256];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n_blocks; i += 256) {
        a += scratch[2 * i];
        b += scratch[2 * i + 1];
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s[0][threadIdx.x] += s[0][threadIdx.x + o];
            s[1][threadIdx.x] += s[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = s[0][0];
        out[1] = s[1][0];
    }
}

}  // namespace vi

namespace {

// Device address of g_energy_scratch. In host code the symbol's name is only a
// host-side stand-in, never a device address, so the address is looked up with
// cudaGetSymbolAddress while the device is current. The lookup is cached per
// device together with the unique id of the CUDA context it was made in: if
// the caller (or another library) resets the device, the next call finds a
// new context, in which the library's module and its static array are loaded
// anew, and looks the address up again instead of writing through the old one.
// The context id comes from the driver's cuCtxGetCurrent / cuCtxGetId, reached
// through the runtime's entry-point query so the library needs no link to
// libcuda; with a driver that lacks them the address is looked up on every
// call.
constexpr int kMaxDevices = 64;
struct ScratchEntry {
    unsigned long long ctx_id;
    void *addr;
};
ScratchEntry g_scratch[kMaxDevices] = {};
std::mutex g_scratch_mutex;

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context (0 when there is none or
// the driver cannot say).
unsigned long long current_ctx_id()
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool queried = false;
    if (!queried) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)f;
        cudaGetLastError();
        queried = true;
    }
    if (!get_current || !get_id)
        return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

cudaError_t scratch_address(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    ScratchEntry &ent = g_scratch[dev];
    const unsigned long long id = current_ctx_id();
    if (!ent.addr || id == 0 || ent.ctx_id != id) {
        void *p = nullptr;
        // binds the device's primary context to this thread if none is
        e = cudaGetSymbolAddress(&p, vi::g_energy_scratch);
        if (e != cudaSuccess)
            return e;
        ent.addr = p;
        ent.ctx_id = current_ctx_id();
    }
    *out = (double *)ent.addr;
    return cudaSuccess;
}

}  // namespace

extern "C" vi_status vi_energy_noalloc(const float *chans_dev, int C, const int32_t *phi_dev,
                                       const uint8_t *code_dev, int W, int H, int T, double *out_dev,
                                       void *cuda_stream)
{
    if (!chans_dev || !phi_dev || !code_dev || !out_dev || (C != 3 && C != 5) || W <= 0 || H <= 0 ||
        T <= 0)
        return VI_ERR_ARG;
    const long long V = (long long)W * H * T;
    if (V > vi::VI_NOALLOC_MAX_VOXELS)
        return VI_ERR_TOO_LARGE;   // more voxels than the static scratch can reduce in one call
    double *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) {
        cudaGetLastError();
        return VI_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int nb = (int)((V + vi::NOALLOC_BLOCK - 1) / vi::NOALLOC_BLOCK);
    VI_COUNT_LAUNCH();
    vi::k_energy_noalloc<<<nb, vi::NOALLOC_BLOCK, 0, st>>>(chans_dev, C, phi_dev, code_dev, W, H, T,
                                                           scratch);
    VI_COUNT_LAUNCH();
    vi::k_energy_noalloc_sum<<<1, 256, 0, st>>>(scratch, nb, out_dev);
    return cudaGetLastError() == cudaSuccess ? VI_OK : VI_ERR_CUDA;
}
