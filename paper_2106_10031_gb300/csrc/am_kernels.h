// am_kernels.h -- launch interface between the host library (am_api.cu) and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "am_common.cuh"

namespace am {

struct MarchArgs {
    const NetDev *nets;
    Arena ar;
    double box, delta;
    int max_n, max_w;        // shared-memory sizing (largest loadable net)
    long long limit;         // persistent schedule: tickets >= limit are not solved
    int64_t begin, end;      // level schedule: cell ids solved by this launch
};
int march_smem_bytes(int max_n, int max_w);
cudaError_t prepare_march_kernels(int max_n, int max_w, int *blocks_per_sm);
// mode 0 = FP64, 1 = double-float (mixed); persistent = ticket queue, else one level [begin, end)
void launch_march(const MarchArgs &a, int mode, bool persistent, int grid, cudaStream_t st);

struct SeedArgs {
    const NetDev *nets;
    Arena ar;
    int net;
    int n_rays;
    const double *origins, *dirs;   // device, n_rays x 3
    double R;
    int max_halvings;
    int max_n, max_w;
    unsigned long long *seed_keys;  // device, n_rays x kw
    double *seed_x;                 // device, n_rays x 3
    int *seed_ok;                   // device, n_rays: 1 ok, -4 no sign change, -5 no common cell
    unsigned long long *n_new;      // device counter of new live seed cells
};
cudaError_t prepare_seed_kernels(int max_n, int max_w);
void launch_seed(const SeedArgs &a, cudaStream_t st);

// ---- mesh assembly
struct AsmArgs {
    Arena ar;
    const NetDev *nets;
    int64_t n_cells;
    int n_nets;
    unsigned long long *face_count;   // n_nets
    unsigned long long *face_fill;    // n_nets
    unsigned long long *face_base;    // n_nets (exclusive scan of face_count)
    unsigned long long *vert_count;   // n_nets
    unsigned long long *vert_base;    // n_nets
    int32_t *perm;                    // faces, grouped by net: cell ids
    int64_t *corner_off;              // faces + 1
    int32_t *corner_vid;              // corners: vertex id local to the net
    unsigned long long *vslots;       // vertex hash table
    unsigned long long vslot_mask;
    double *out_xyz;                  // 3 x vertices
    int32_t *out_fv;                  // corners
    int32_t *out_edges;               // corners
    unsigned long long *out_keys;     // faces x kw
    int64_t n_faces;
};
void launch_asm_count(const AsmArgs &a, cudaStream_t st);
void launch_asm_scatter(const AsmArgs &a, cudaStream_t st);
cudaError_t launch_asm_offsets(const AsmArgs &a, int64_t *scan_tmp, int64_t scan_tmp_len, cudaStream_t st);
void launch_asm_vertices(const AsmArgs &a, cudaStream_t st);
void launch_asm_lookup(const AsmArgs &a, cudaStream_t st);
void launch_asm_write(const AsmArgs &a, cudaStream_t st);

}  // namespace am
