// Level-set extraction from a phi grid by marching tetrahedra (the offset
// surfaces of Sec. 6: the c-level set of phi sampled on a grid).
//
// Every cube of the grid is split into the six tetrahedra of its Kuhn
// triangulation (for each permutation of the axes, the path 000 -> e_a ->
// e_a + e_b -> 111), which splits shared faces the same way in both cubes, so
// the surface is watertight without the case ambiguities of marching cubes.
// Every edge of the triangulation runs from a node to node + d, d one of
// x, y, z, xy, xz, yz, xyz (numbered 0..6); a cut edge (exactly one end with
// phi < level) carries one vertex at the linear interpolation point, and the
// vertices are numbered by (node, direction).  Triangles come cube by cube,
// tetrahedra in the permutation order (x,y,z), (x,z,y), (y,x,z), (y,z,x),
// (z,x,y), (z,y,x); a tetrahedron with two inside corners i, j and two
// outside k, l (path order) gives the quad ik, il, jl, jk split along ik-jl.
// Orientation (normals from phi < level towards phi >= level) is
// combinatorial: the six tetrahedra alternate in orientation, and on a
// positively oriented one (v0, v1, v2, v3) a lone inside corner i gives the
// triangle (ix, iy, iz) for (i, x, y, z) an even permutation of the corners.
//
// Passes (all deterministic): per node the mask of cut edges and its count;
// exclusive scan -> vertex numbers; vertices; per cube the triangle count;
// scan -> triangle offsets; triangles.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "internal.h"

namespace ptsdf {

namespace {

constexpr int kMeshThreads = 256;

struct Grid {
    const float* phi;
    int nx, ny, nz;
    float ox, oy, oz, hx, hy, hz;
    float level;
};

// corner bit pattern (x = 1, y = 2, z = 4) of each Kuhn tetrahedron's path
__constant__ uint8_t c_tet[6][4] = {{0, 1, 3, 7}, {0, 1, 5, 7}, {0, 2, 3, 7}, {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 6, 7}};
// orientation of each (sign of det[v1 - v0, v2 - v0, v3 - v0])
__constant__ int8_t c_tet_sign[6] = {1, -1, -1, 1, 1, -1};
// direction number of an edge from corner bits u to v (u a subset of v), by v ^ u
__constant__ int8_t c_dir_of_diff[8] = {-1, 0, 1, 3, 2, 4, 5, 6};
// for corner i of a tetrahedron, the other three in the order that makes
// (i, x, y, z) an even permutation of (0, 1, 2, 3)
__constant__ int8_t c_even[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
// node offsets of the 7 directions
__constant__ int8_t c_dir_off[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};

__device__ __forceinline__ int64_t node_index(const Grid& g, int i, int j, int k) {
    return ((int64_t)k * g.ny + j) * g.nx + i;
}

__device__ __forceinline__ bool inside_at(const Grid& g, int i, int j, int k) {
    return g.phi[node_index(g, i, j, k)] < g.level;
}

__global__ void k_mt_edges(Grid g, uint8_t* __restrict__ mask, int32_t* __restrict__ cnt) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)g.nx * g.ny * g.nz;
    if (n >= total) return;
    const int i = (int)(n % g.nx), j = (int)((n / g.nx) % g.ny), k = (int)(n / ((int64_t)g.nx * g.ny));
    const bool in0 = inside_at(g, i, j, k);
    unsigned m = 0;
    for (int d = 0; d < 7; ++d) {
        const int a = i + c_dir_off[d][0], b = j + c_dir_off[d][1], c = k + c_dir_off[d][2];
        if (a >= g.nx || b >= g.ny || c >= g.nz) continue;
        if (inside_at(g, a, b, c) != in0) m |= 1u << d;
    }
    mask[n] = (uint8_t)m;
    cnt[n] = __popc(m);
}

__global__ void k_mt_verts(Grid g, const uint8_t* __restrict__ mask, const int32_t* __restrict__ off,
                           float* __restrict__ verts) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)g.nx * g.ny * g.nz;
    if (n >= total) return;
    const unsigned m = mask[n];
    if (!m) return;
    const int i = (int)(n % g.nx), j = (int)((n / g.nx) % g.ny), k = (int)(n / ((int64_t)g.nx * g.ny));
    const float pa = g.phi[n];
    int32_t v = off[n];
    for (int d = 0; d < 7; ++d) {
        if (!(m & (1u << d))) continue;
        const int di = c_dir_off[d][0], dj = c_dir_off[d][1], dk = c_dir_off[d][2];
        const float pb = g.phi[node_index(g, i + di, j + dj, k + dk)];
        const float t = (g.level - pa) / (pb - pa);
        verts[3 * (int64_t)v] = g.ox + g.hx * ((float)i + t * (float)di);
        verts[3 * (int64_t)v + 1] = g.oy + g.hy * ((float)j + t * (float)dj);
        verts[3 * (int64_t)v + 2] = g.oz + g.hz * ((float)k + t * (float)dk);
        ++v;
    }
}

__device__ __forceinline__ unsigned cube_inside_bits(const Grid& g, int i, int j, int k) {
    unsigned b = 0;
    for (int c = 0; c < 8; ++c)
        if (inside_at(g, i + (c & 1), j + ((c >> 1) & 1), k + ((c >> 2) & 1))) b |= 1u << c;
    return b;
}

__global__ void k_mt_tcount(Grid g, int32_t* __restrict__ cnt) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int cx = g.nx - 1, cy = g.ny - 1;
    const int64_t total = (int64_t)cx * cy * (g.nz - 1);
    if (c >= total) return;
    const int i = (int)(c % cx), j = (int)((c / cx) % cy), k = (int)(c / ((int64_t)cx * cy));
    const unsigned bits = cube_inside_bits(g, i, j, k);
    int t = 0;
    if (bits != 0 && bits != 0xffu) {
        for (int q = 0; q < 6; ++q) {
            int nin = 0;
            for (int v = 0; v < 4; ++v) nin += (bits >> c_tet[q][v]) & 1u;
            t += (nin == 1 || nin == 3) ? 1 : (nin == 2 ? 2 : 0);
        }
    }
    cnt[c] = t;
}

// vertex number of the cut edge between cube corners u and v (bit patterns)
__device__ __forceinline__ int32_t edge_vertex(const Grid& g, const uint8_t* __restrict__ mask,
                                               const int32_t* __restrict__ voff, int i, int j, int k, int u, int v) {
    const int lo = (u & v) == u ? u : v;   // the corner whose bits the other's contain
    const int hi = lo == u ? v : u;
    const int d = c_dir_of_diff[hi ^ lo];
    const int64_t n = node_index(g, i + (lo & 1), j + ((lo >> 1) & 1), k + ((lo >> 2) & 1));
    return voff[n] + __popc((unsigned)mask[n] & ((1u << d) - 1u));
}

__global__ void k_mt_tris(Grid g, const uint8_t* __restrict__ mask, const int32_t* __restrict__ voff,
                          const int32_t* __restrict__ toff, int32_t* __restrict__ tris) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int cx = g.nx - 1, cy = g.ny - 1;
    const int64_t total = (int64_t)cx * cy * (g.nz - 1);
    if (c >= total) return;
    const int i = (int)(c % cx), j = (int)((c / cx) % cy), k = (int)(c / ((int64_t)cx * cy));
    const unsigned bits = cube_inside_bits(g, i, j, k);
    if (bits == 0 || bits == 0xffu) return;
    int64_t out = toff[c];
    auto emit = [&](int a0, int a1, int b0, int b1, int c0, int c1, bool flip) {
        const int32_t va = edge_vertex(g, mask, voff, i, j, k, a0, a1);
        const int32_t vb = edge_vertex(g, mask, voff, i, j, k, b0, b1);
        const int32_t vc = edge_vertex(g, mask, voff, i, j, k, c0, c1);
        tris[3 * out] = va;
        tris[3 * out + 1] = flip ? vc : vb;
        tris[3 * out + 2] = flip ? vb : vc;
        ++out;
    };
    for (int q = 0; q < 6; ++q) {
        int cv[4], in[4], nin = 0;
        for (int v = 0; v < 4; ++v) {
            cv[v] = c_tet[q][v];
            in[v] = (bits >> cv[v]) & 1u;
            nin += in[v];
        }
        if (nin == 0 || nin == 4) continue;
        const bool neg = c_tet_sign[q] < 0;
        if (nin == 1 || nin == 3) {
            // the lone corner and the even permutation starting with it
            int lone = 0;
            for (int v = 0; v < 4; ++v)
                if ((in[v] != 0) == (nin == 1)) lone = v;
            const int x = c_even[lone][0], y = c_even[lone][1], z = c_even[lone][2];
            // outward for a lone inside corner on a positive tetrahedron; reversed for a
            // lone outside corner and for a negative tetrahedron
            const bool flip = (nin == 3) != neg;
            emit(cv[lone], cv[x], cv[lone], cv[y], cv[lone], cv[z], flip);
        } else {
            int ii[2], oo[2], a = 0, b = 0;
            for (int v = 0; v < 4; ++v) {
                if (in[v]) ii[a++] = v;
                else oo[b++] = v;
            }
            // parity of (i, j, k, l) as a permutation of (0, 1, 2, 3)
            const int p[4] = {ii[0], ii[1], oo[0], oo[1]};
            int inv = 0;
            for (int s = 0; s < 4; ++s)
                for (int t = s + 1; t < 4; ++t) inv += p[s] > p[t];
            const bool flip = ((inv & 1) != 0) != neg;
            const int I = cv[ii[0]], J = cv[ii[1]], K = cv[oo[0]], L = cv[oo[1]];
            emit(I, K, I, L, J, L, flip);   // (ik, il, jl)
            emit(I, K, J, L, J, K, flip);   // (ik, jl, jk)
        }
    }
}

// exclusive scan of n int32 values in place; returns the total
__global__ void k_scan_blocks(int32_t* __restrict__ v, int64_t n, int64_t* __restrict__ block_sum) {
    __shared__ int64_t s[kMeshThreads];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t x = i < n ? v[i] : 0;
    s[threadIdx.x] = x;
    __syncthreads();
    for (int off = 1; off < kMeshThreads; off <<= 1) {
        const int64_t y = threadIdx.x >= (unsigned)off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += y;
        __syncthreads();
    }
    if (i < n) v[i] = (int32_t)(s[threadIdx.x] - x);
    if (threadIdx.x == kMeshThreads - 1) block_sum[blockIdx.x] = s[threadIdx.x];
}

__global__ void k_add_block_offsets(int32_t* __restrict__ v, int64_t n, const int64_t* __restrict__ block_off) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] += (int32_t)block_off[blockIdx.x];
}

cudaError_t exclusive_scan(int32_t* d_v, int64_t n, int64_t* total, cudaStream_t st) {
    const int64_t blocks = (n + kMeshThreads - 1) / kMeshThreads;
    int64_t* d_bs = nullptr;
    cudaError_t e = cudaMallocAsync(&d_bs, (size_t)blocks * sizeof(int64_t), st);
    if (e != cudaSuccess) return e;
    k_scan_blocks<<<(unsigned)blocks, kMeshThreads, 0, st>>>(d_v, n, d_bs);
    e = cudaGetLastError();
    std::vector<int64_t> h((size_t)blocks);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d_bs, (size_t)blocks * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
        int64_t run = 0;
        for (auto& x : h) {
            const int64_t y = x;
            x = run;
            run += y;
        }
        *total = run;
        e = cudaMemcpyAsync(d_bs, h.data(), (size_t)blocks * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) {
        k_add_block_offsets<<<(unsigned)blocks, kMeshThreads, 0, st>>>(d_v, n, d_bs);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // h must outlive the copy
    cudaFreeAsync(d_bs, st);
    return e;
}

}  // namespace

}  // namespace ptsdf

using namespace ptsdf;

extern "C" sdf_status sdf_mesh_level_set(const float* d_phi, int32_t nx, int32_t ny, int32_t nz, const float* origin,
                                         const float* spacing, float level, float* d_vertices, int64_t cap_vertices,
                                         int32_t* d_triangles, int64_t cap_triangles, int64_t* n_vertices,
                                         int64_t* n_triangles, void* stream) {
    if (!d_phi || !origin || !spacing || !n_vertices || !n_triangles)
        return set_error(SDF_EINVAL, "sdf_mesh_level_set: NULL argument");
    if (nx < 2 || ny < 2 || nz < 2) return set_error(SDF_EINVAL, "sdf_mesh_level_set: need at least 2 nodes per axis");
    const int64_t nodes = (int64_t)nx * ny * nz;
    if (nodes > (int64_t)1 << 31) return set_error(SDF_EINVAL, "sdf_mesh_level_set: more than 2^31 nodes");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Grid g{d_phi, nx, ny, nz, origin[0], origin[1], origin[2], spacing[0], spacing[1], spacing[2], level};
    const int64_t cubes = (int64_t)(nx - 1) * (ny - 1) * (nz - 1);
    uint8_t* mask = nullptr;
    int32_t *voff = nullptr, *toff = nullptr;
    cudaError_t e = cudaMallocAsync(&mask, (size_t)nodes, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&voff, (size_t)nodes * sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&toff, (size_t)cubes * sizeof(int32_t), st);
    int64_t nv = 0, nt = 0;
    sdf_status s = SDF_OK;
    if (e == cudaSuccess) {
        k_mt_edges<<<(unsigned)((nodes + kMeshThreads - 1) / kMeshThreads), kMeshThreads, 0, st>>>(g, mask, voff);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = exclusive_scan(voff, nodes, &nv, st);
    if (e == cudaSuccess) {
        k_mt_tcount<<<(unsigned)((cubes + kMeshThreads - 1) / kMeshThreads), kMeshThreads, 0, st>>>(g, toff);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = exclusive_scan(toff, cubes, &nt, st);
    if (e == cudaSuccess) {
        *n_vertices = nv;
        *n_triangles = nt;
        if (nv >= ((int64_t)1 << 31) || nt >= ((int64_t)1 << 31)) {
            s = set_error(SDF_EINVAL, "sdf_mesh_level_set: more than 2^31 vertices or triangles");
        } else if (d_vertices || d_triangles) {
            if (!d_vertices || !d_triangles || cap_vertices < nv || cap_triangles < nt) {
                s = set_error(SDF_EINVAL, "sdf_mesh_level_set: output buffers missing or too small");
            } else {
                k_mt_verts<<<(unsigned)((nodes + kMeshThreads - 1) / kMeshThreads), kMeshThreads, 0, st>>>(
                    g, mask, voff, d_vertices);
                e = cudaGetLastError();
                if (e == cudaSuccess) {
                    k_mt_tris<<<(unsigned)((cubes + kMeshThreads - 1) / kMeshThreads), kMeshThreads, 0, st>>>(
                        g, mask, voff, toff, d_triangles);
                    e = cudaGetLastError();
                }
            }
        }
    }
    cudaFreeAsync(mask, st);
    cudaFreeAsync(voff, st);
    cudaFreeAsync(toff, st);
    if (s != SDF_OK) return s;
    return e == cudaSuccess ? SDF_OK : cuda_error(e, "sdf_mesh_level_set");
}
