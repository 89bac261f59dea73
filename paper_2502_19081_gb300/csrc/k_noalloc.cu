// Neighbour-list build that allocates nothing: the same cell-list and
// neighbour kernels as the context path, with their scratch (a folded copy of
// the positions, the cell list, the status words, the reference positions)
// held in a file-scope device array instead of a caller workspace.
//
// Who needs it: code that is not allowed to call cudaMalloc -- a plugin inside
// a host program that owns every device allocation through its own pool, or a
// loop that cannot afford the implicit device synchronisation of an
// allocation.  Such a caller passes its own input and output buffers; the
// scratch below is reserved once when the library is loaded on a device and
// stays reserved until the process exits.
#include <cstring>
#include <mutex>

#include "mix_launch.h"

namespace mixd {

namespace {

constexpr int64_t NA_MAX_ATOMS = MIX_NOALLOC_MAX_ATOMS;
constexpr int64_t NA_MAX_CELLS = MIX_NOALLOC_MAX_CELLS;

constexpr size_t na_al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t NA_O_STATUS = 0;
constexpr size_t NA_O_X = na_al(NA_O_STATUS + SW_COUNT * sizeof(int));
constexpr size_t NA_O_XB = na_al(NA_O_X + NA_MAX_ATOMS * sizeof(double4));
constexpr size_t NA_O_XF = na_al(NA_O_XB + NA_MAX_ATOMS * sizeof(double4));
constexpr size_t NA_O_XR = na_al(NA_O_XF + NA_MAX_ATOMS * sizeof(float4));
constexpr size_t NA_O_CELL3 = na_al(NA_O_XR + NA_MAX_ATOMS * sizeof(float4));
constexpr size_t NA_O_CELL_OF = na_al(NA_O_CELL3 + NA_MAX_ATOMS * sizeof(int));
constexpr size_t NA_O_CELL_ATOMS = na_al(NA_O_CELL_OF + NA_MAX_ATOMS * sizeof(int));
constexpr size_t NA_O_CELL_COUNT = na_al(NA_O_CELL_ATOMS + NA_MAX_ATOMS * sizeof(int));
constexpr size_t NA_O_CELL_FILL = na_al(NA_O_CELL_COUNT + NA_MAX_CELLS * sizeof(int));
constexpr size_t NA_O_CELL_START = na_al(NA_O_CELL_FILL + NA_MAX_CELLS * sizeof(int));
constexpr size_t NA_BYTES = na_al(NA_O_CELL_START + (NA_MAX_CELLS + 1) * sizeof(int));

// the scratch; every GPU that loads the library holds it until exit
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
unsigned char* g_na_ptr[NA_MAX_DEVICES] = {};

// Zero what must start at zero (status words, cell counts) and request a build.
__global__ void k_noalloc_init(int* status, int* cell_count, int ncell) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < SW_COUNT) status[t] = (t == SW_REBUILD) ? 1 : 0;
    for (int k = t; k < ncell; k += gridDim.x * blockDim.x) cell_count[k] = 0;
}

// The position checks the context path makes before a build: a non-finite
// coordinate, or one outside a non-periodic dimension of the box, sets its
// status bit (the build still runs; every cell index it forms is clamped).
__global__ void k_noalloc_check(Dev d) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.n; i += (int64_t)gridDim.x * blockDim.x) {
        const double4 x = d.x[i];
        if (!(isfinite(x.x) && isfinite(x.y) && isfinite(x.z))) {
            set_status(d.status, ST_NONFINITE);
            continue;
        }
        const double xs[3] = {x.x, x.y, x.z};
        for (int k = 0; k < 3; ++k)
            if (!d.box.per[k] && (xs[k] < d.box.lo[k] || xs[k] >= d.box.lo[k] + d.box.L[k]))
                set_status(d.status, ST_OUT_OF_BOX);
    }
}

// Device address of the scratch on the current device, looked up once per device.
int scratch_address(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return MIX_ECUDA;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MIX_ECUDA;
        g_na_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_na_ptr[dev];
    return MIX_OK;
}

}  // namespace
}  // namespace mixd

using namespace mixd;

extern "C" int mix_neighbours_noalloc(int64_t n_atoms, const double* x_dev, const double* box_lo,
                                      const double* box_len, const int* periodic, double r_list, int cap,
                                      int* nnb_dev, int* nbr_dev, int* rev_dev, void* cuda_stream) {
    if (n_atoms < 0 || n_atoms > NA_MAX_ATOMS) return MIX_EINVAL;
    if (!box_lo || !box_len || !periodic || !(r_list > 0) || cap < 1 || cap > MAX_CAP) return MIX_EINVAL;
    if (n_atoms > 0 && (!x_dev || !nnb_dev || !nbr_dev || !rev_dev)) return MIX_EINVAL;
    if ((uintptr_t)x_dev & 15) return MIX_EINVAL;
    Dev d;
    memset(&d, 0, sizeof d);
    d.n = n_atoms;
    d.cap = cap;
    int64_t ncell = 1;
    for (int k = 0; k < 3; ++k) {
        if (!(box_len[k] > 0)) return MIX_EINVAL;
        d.box.lo[k] = box_lo[k];
        d.box.L[k] = box_len[k];
        d.box.invL[k] = 1.0 / box_len[k];
        d.box.per[k] = periodic[k] ? 1 : 0;
        // the cell count is checked as a double before it becomes an int
        const double ratio = box_len[k] / r_list;
        if (!(ratio < 1024.0)) return MIX_EINVAL;
        int nc = (int)floor(ratio);
        if (d.box.per[k]) {
            if (box_lo[k] != 0.0 || nc < 3 || box_len[k] < 2.0 * r_list) return MIX_EINVAL;
        } else if (nc < 1) {
            nc = 1;
        }
        d.cells.nc[k] = nc;
        d.cells.invh[k] = (double)nc / box_len[k];
        d.cells.h[k] = box_len[k] / (double)nc;
        d.cells.hf[k] = (float)d.cells.h[k];
        if (nc > 1023) return MIX_EINVAL;
        ncell *= nc;
    }
    if (ncell > NA_MAX_CELLS) return MIX_EINVAL;
    d.cells.ncell = (int)ncell;
    d.rlist2 = r_list * r_list;
    unsigned char* base = nullptr;
    int st = scratch_address(&base);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    d.status = reinterpret_cast<int*>(base + NA_O_STATUS);
    d.x = reinterpret_cast<double4*>(base + NA_O_X);
    d.xb = reinterpret_cast<double4*>(base + NA_O_XB);
    d.xf = reinterpret_cast<float4*>(base + NA_O_XF);
    d.xr = reinterpret_cast<float4*>(base + NA_O_XR);
    d.cell3 = reinterpret_cast<int*>(base + NA_O_CELL3);
    double extent = 0.0;
    for (int k = 0; k < 3; ++k) extent = fmax(extent, fabs(box_lo[k]) + box_len[k]);
    d.exact_lists = extent > 2000.0 ? 1 : 0;
    d.cell_of = reinterpret_cast<int*>(base + NA_O_CELL_OF);
    d.cell_atoms = reinterpret_cast<int*>(base + NA_O_CELL_ATOMS);
    d.cell_count = reinterpret_cast<int*>(base + NA_O_CELL_COUNT);
    d.cell_fill = reinterpret_cast<int*>(base + NA_O_CELL_FILL);
    d.cell_start = reinterpret_cast<int*>(base + NA_O_CELL_START);
    d.nnb = nnb_dev;
    d.nbr = nbr_dev;
    d.rev = rev_dev;
    if (n_atoms > 0 &&
        cudaMemcpyAsync(d.x, x_dev, (size_t)n_atoms * sizeof(double4), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return MIX_ECUDA;
    k_noalloc_init<<<64, 256, 0, s>>>(d.status, d.cell_count, d.cells.ncell);
    if (n_atoms > 0) k_noalloc_check<<<(int)((n_atoms + 255) / 256), 256, 0, s>>>(d);
    launch_build(d, s);
    if (cudaGetLastError() != cudaSuccess) return MIX_ECUDA;
    int status[SW_COUNT];
    if (cudaMemcpyAsync(status, d.status, sizeof status, cudaMemcpyDeviceToHost, s) != cudaSuccess) return MIX_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MIX_ECUDA;
    if (status[SW_STATUS] & ST_NONFINITE) return MIX_ENUMERIC;
    if (status[SW_STATUS] & ST_OUT_OF_BOX) return MIX_EBOX;
    if (status[SW_STATUS] & ST_NBR_OVERFLOW) return MIX_EOVERFLOW;
    if (status[SW_STATUS] & ST_REV_MISSING) return MIX_EINVAL;
    return MIX_OK;
}
