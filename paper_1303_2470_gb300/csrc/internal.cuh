// internal.cuh -- declarations shared by the translation units of libmp (not part of the
// C ABI). Lattice constants, the packed geometry, error reporting and kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>

#include "../../include/mp.h"

namespace mp {

// ---------------------------------------------------------------------------------------
// D3Q19 velocity set, ordered by the z component of c: rest, the 8 in-plane links, the 5
// links with c_z = +1, the 5 links with c_z = -1. Weights 1/3 (rest), 1/18 (|c| = 1) and
// 1/36 (|c| = sqrt 2). Lookups are meant for fully unrolled loops, where they fold to
// immediates.
// ---------------------------------------------------------------------------------------
constexpr int kQ = 19;

__host__ __device__ constexpr int cx(int i)
{
    constexpr int t[kQ] = {0, 1, -1, 0, 0, 1, -1, 1, -1, 0, 1, -1, 0, 0, 0, 1, -1, 0, 0};
    return t[i];
}
__host__ __device__ constexpr int cy(int i)
{
    constexpr int t[kQ] = {0, 0, 0, 1, -1, 1, -1, -1, 1, 0, 0, 0, 1, -1, 0, 0, 0, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int cz(int i)
{
    constexpr int t[kQ] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, -1, -1, -1, -1, -1};
    return t[i];
}
__host__ __device__ constexpr int ci(int i, int g) { return g == 0 ? cx(i) : (g == 1 ? cy(i) : cz(i)); }
__host__ __device__ constexpr int opposite(int i)
{
    constexpr int t[kQ] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 14, 16, 15, 18, 17, 9, 11, 10, 13, 12};
    return t[i];
}
__host__ __device__ constexpr bool is_face(int i) { return (cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i)) == 1; }
template <typename T>
__host__ __device__ constexpr T weight(int i)
{
    return i == 0 ? T(1) / T(3) : (is_face(i) ? T(1) / T(18) : T(1) / T(36));
}

// ---------------------------------------------------------------------------------------
// Packed geometry on the device. Bits are per 32 consecutive nodes (linear order):
// word w covers nodes 32w .. 32w+31, bit b = node 32w+b.
//   fluid[w]  bit set = fluid node
//   iface[w]  bit set = interfacial fluid node (>= 1 solid D3Q19 neighbour)
//   ibase[w]  number of interfacial nodes before node 32w (exclusive prefix), so the
//             compact index of interfacial node n is ibase[n>>5] + popc(iface[n>>5] & lt)
//   ilist[k]  node index of the k-th interfacial node, increasing
//   fbase[w], flist[k]  the same prefix and list for all fluid nodes (work list of the MP)
// ---------------------------------------------------------------------------------------
struct Geometry {
    int nx = 0, ny = 0, nz = 0;
    int N = 0;  // nodes
    int W = 0;  // words
    int64_t n_fluid = 0, n_iface = 0;
    uint32_t* fluid = nullptr;
    uint32_t* iface = nullptr;
    int32_t* ibase = nullptr;
    int32_t* ilist = nullptr;
    int32_t* fbase = nullptr;
    int32_t* flist = nullptr;
    uint32_t* cluster = nullptr;  // bit set = node of the largest connected fluid cluster
    int64_t n_cluster = 0;
};

// Launch with programmatic dependent launch allowed: on the same stream the kernel may start
// while the previous kernel drains (its blocks become resident and wait). Such a kernel calls
// pdl_enter() first: it lets its own dependents start, then waits until the previous grid has
// finished and its writes are visible, so nothing it reads or writes can race with it.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

__device__ __forceinline__ void pdl_enter()
{
    cudaTriggerProgrammaticLaunchCompletion();
    cudaGridDependencySynchronize();
}

// Error reporting: the thread-local last-error text behind mp_last_error().
void set_error(const std::string& msg);
void clear_error();
int cuda_fail(cudaError_t e, const char* what);

#define MP_CUDA(call)                                          \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return mp::cuda_fail(e_, #call); \
    } while (0)

// Geometry prep (geometry.cu): validates the mask, classifies nodes and builds the packed
// arrays above on `stream` (the two node lists only when `want_list`). Allocates with cudaMallocAsync on the stream when
// `stream_ordered`, else with cudaMalloc. Synchronises the stream (counts go to the host).
int build_geometry(const mp_geometry* g, cudaStream_t stream, bool stream_ordered,
                   bool want_list, Geometry* out);
void free_geometry(Geometry* g, cudaStream_t stream, bool stream_ordered);

// Largest connected cluster of fluid nodes (D3Q19 links, periodic) into g->cluster and
// g->n_cluster; ties go to the cluster holding the smallest node index. Synchronises.
int build_cluster(Geometry* g, cudaStream_t stream, bool stream_ordered);

}  // namespace mp
