// idp_remesh.h -- host interface of the device re-mesher (k_remesh.cu): the
// adaptation plan of one mesh and the mesh tables of the adapted leaves,
// built on the device into caller-provided buffers.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "idp_device.cuh"

namespace idp {

// the level-0 grid, box and boundary kinds (0 = periodic) of the mesh
struct RemeshMesh {
    int nx0, ny0;
    double x0, y0, x1, y1;
    int bc[4];
};

// plan: the current leaves and their connectivity (device arrays)
struct PlanIn {
    int K;
    const double *ind;
    const int8_t *lev;
    const int *ix, *iy;
    const int4 *fnbr;
    const uchar4 *ftype;
    const int32_t *m_large;
    const int2 *m_small;
    double refine, coarsen;
    int min_level, max_level;
};
// the adapted leaves in the plan's order, with their transfer kind and
// sources (as idp_amr_plan) and the transfer's families (as idp_amr_transfer
// forms them); capacity: the entries the buffers hold
struct PlanOut {
    int capacity;
    int8_t *lev;
    int *ix, *iy, *kind;
    int4 *src, *fam;
};

struct BuildIn {
    RemeshMesh mesh;
    int K;
    const int8_t *lev;
    const int *ix, *iy;
};
struct BuildOut {
    Geo *geom;
    GeoC *geoc;
    int *sim;
    int4 *fnbr;
    uchar4 *ftype;
    int32_t *m_large;
    int2 *m_small;
    int32_t *m_info;
    int capM;
};

struct NodesIn {
    int NP, K, M, W;
    const int32_t *m_large;
    const int2 *m_small;
    const int32_t *m_info;
};
struct NodesOut {
    int32_t *mn_node;
    int2 *mn_slot;
    int32_t *mb_node_off, *mb_for_off, *mb_foreign;
    int cap_nodes, cap_foreign, cap_blocks;
};

size_t remesh_plan_scratch_ints(int K);
// K_new: the adapted leaf count (nothing is written when it exceeds
// out.capacity); n_fam: the families; iterations: balance sweeps (-1 and
// nothing written when 64 sweeps did not reach the fixed point)
cudaError_t remesh_plan(const PlanIn &in, PlanOut &out, int *scratch, cudaStream_t st, int num_sms, int *K_new,
                        int *n_fam, int *iterations);
size_t remesh_build_scratch_bytes(int K, int NP);
// faces and mortars; M_new: the mortars (not written beyond out.capM);
// err_bits: 1 duplicate leaf, 2 not 2:1 balanced, 4 a small side without
// its mortar
cudaError_t remesh_build_faces(const BuildIn &in, BuildOut &out, void *scratch, cudaStream_t st, int num_sms,
                               int *M_new, int *err_bits);
size_t remesh_nodes_scratch_bytes(int K, int NP, int M, int W);
// mortar nodes and limiting blocks; err_bits: 8 a node on three mortars,
// 16 a block with too many foreign mortars
cudaError_t remesh_build_mortar_nodes(const NodesIn &in, NodesOut &out, void *scratch, cudaStream_t st, int num_sms,
                                      int *n_mnodes, int *n_blocks, int *fmax, int *err_bits);

// out[0] = the leaves' area, out[1] = the mortars' large-face length (device,
// asynchronous; a fixed summation order)
void remesh_totals(const RemeshMesh &mesh, const int8_t *lev, int K, const int32_t *m_large, const int32_t *m_info,
                   int M, double *out, cudaStream_t st);

}  // namespace idp
