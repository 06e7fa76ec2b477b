// grid.h -- launchers of grid.cu (sparse leaf tables, instance construction, fusion).
#pragma once

#include "internal.h"

namespace vgp {

struct Table {
    uint64_t* keys = nullptr;
    uint32_t mask = 0;
    size_t cap() const { return keys ? (size_t)mask + 1 : 0; }
};

// fused surface properties of the global grid (Eq. 6, Sec. IV-C): per pool voxel nc channels
// and one variance (weight for Eq. 9); W = NaN: no property fused yet
struct PropGrid {
    double* C = nullptr;
    double* W = nullptr;
    int nc = 0;
};
// one frame's property estimates by testing voxel
struct PropIn {
    const double* c = nullptr;
    const double* w = nullptr;
    int nc = 0;
};

void collect_table(const Table& t, int32_t* slot2idx, int32_t* list, uint64_t* keys_out, int* count_dev,
                   int64_t list_cap, int* err, cudaStream_t st);

// frame (L-GPDF)
void frame_voxelise(const float* pts, int64_t n, const DevParams& P, const Table& t, unsigned long long* masks,
                    int* n_valid, int* err, cudaStream_t st);
void frame_leaf_counts(const int32_t* list, int nl, const unsigned long long* masks, int cap, int32_t* nocc,
                       int64_t* ninst, cudaStream_t st);
void frame_leaf_points(const int32_t* list, const uint64_t* lkeys, int nl, const unsigned long long* masks,
                       const int32_t* nocc, const int64_t* inst_off, const DevParams& P, double* X, double* Xl,
                       float* Xf, char4* Xi, double* centre, cudaStream_t st);
void frame_dilate(const uint64_t* lkeys, int nl, const Table& t, int* err, cudaStream_t st);
void frame_assign_tests(const uint64_t* tl_keys, int ntl, const Table& ft, const int32_t* slot2leaf,
                        int64_t* inst_cnt, int* n_orphan, cudaStream_t st);
void frame_scatter_tests(const uint64_t* tl_keys, int ntl, const Table& ft, const int32_t* slot2leaf,
                         const int64_t* q_off, int64_t* cursor, uint64_t* tkey, cudaStream_t st);

// ray-cast testing points (Sec. IV-B)
void frame_surface_voxels(const int32_t* list, const uint64_t* lkeys, int nl, const unsigned long long* masks,
                          const int64_t* soff, uint64_t* svox, cudaStream_t st);
void frame_raycast_tests(const uint64_t* svox, int64_t ns, const Table& ft, const unsigned long long* fmasks,
                         const Table& g, const int32_t* g_slot2pool, const unsigned long long* g_known,
                         const double origin[3], int have_o, const int ov[3], double vs, int K, const Table& tt,
                         unsigned* tflags, int* err, cudaStream_t st);
void frame_collect_tests(const Table& tt, const unsigned* tflags, uint64_t* out_key, int8_t* out_sign, int* count,
                         cudaStream_t st);
void frame_assign_list(const uint64_t* tkey, int64_t nt, const Table& ft, const int32_t* slot2leaf, int R,
                       int32_t* tinst, int64_t* inst_cnt, int* n_orphan, cudaStream_t st);
void frame_scatter_list(const uint64_t* tkey, const int8_t* tsign, int64_t nt, const int32_t* tinst, const int64_t* q_off,
                        int64_t* cursor, int64_t orphan_base, int* orphan_cursor, uint64_t* gkey, int8_t* gsign,
                        cudaStream_t st);
void frame_orphans_and_sign(int64_t nt, int64_t n_assigned, const int8_t* sign, double* d, double* grad, double* v,
                            uint8_t* status, cudaStream_t st);

// surface (G-GPDF)
void surface_bin(const float* pts, int64_t n, const DevParams& P, const Table& t, int32_t* pt_slot, int32_t* slot_cnt,
                 int* n_valid, int* err, cudaStream_t st);
void surface_leaf_counts(const int32_t* list, int nl, const int32_t* slot_cnt, int64_t* cnt, cudaStream_t st);
void surface_scatter(const int32_t* pt_slot, int64_t n, const int32_t* slot2leaf, const int64_t* off, int32_t* cursor,
                     int32_t* idx, int nl, cudaStream_t st);

// queries
void query_leaf(const float* q, int64_t n, const DevParams& P, const Table& t, int32_t* q_slot, int* err,
                cudaStream_t st);
void group_centre(const uint64_t* gkeys, int ng, const Table& s, int R, uint64_t* gcen, cudaStream_t st);
void insert_centres(const uint64_t* gcen, int ng, const Table& it, int* err, cudaStream_t st);
void inst_count(const uint64_t* ikey, int ni, const Table& s, const int32_t* sslot2leaf, const int64_t* soff, int cap,
                int64_t* ncand, int64_t* ninst, cudaStream_t st, int single = 0);
void inst_gather(const uint64_t* ikey, int ni, const Table& s, const int32_t* sslot2leaf, const int64_t* soff,
                 const int32_t* sidx, const float* spts, const int64_t* ncand, const int64_t* inst_off,
                 const DevParams& P, double* Xl, float* Xf, int64_t* gidx, double* centre, cudaStream_t st,
                 int single = 0);

// G-GPDF blended per-leaf GPs (Eq. 10)
void smooth_nodes(const uint64_t* gcen, int ng, const Table& s, const Table& it, int* err, cudaStream_t st);
void smooth_pairs(const float* q, int64_t n, const int32_t* q_slot, const int32_t* slot2group, const uint64_t* gcen,
                  const Table& s, const Table& it, const int32_t* islot2inst, const DevParams& P, int Q,
                  int32_t* pair_inst, uint8_t* n_nodes, int64_t* inst_cnt, cudaStream_t st);
void smooth_scatter(const int32_t* pair_inst, int64_t npairs, const int64_t* q_off, int64_t* cursor, int64_t* qidx,
                    cudaStream_t st);
void smooth_blend(int64_t n, int Q, const int32_t* q_slot, const uint8_t* n_nodes, const double* pd, const double* pg,
                  const double* pv, const uint8_t* ps, double lambda, const DevParams& P, double* d, double* grad,
                  double* var, uint8_t* status, cudaStream_t st);
void query_route(const int32_t* q_slot, int64_t n, const int32_t* slot2group, const uint64_t* gcen, const Table& it,
                 const int32_t* islot2inst, int32_t* q_inst, int64_t* inst_qcnt, cudaStream_t st);
void query_scatter(const int32_t* q_inst, int64_t n, const int64_t* q_off, int64_t* cursor, int64_t* qidx, double* d,
                   double* grad, double* var, uint8_t* status, cudaStream_t st);

// fusion, export, import
void fuse_clear_flags(int32_t* flags, int n, cudaStream_t st);
void fuse_insert(const uint64_t* vkey, const double* d, const double* v, const uint8_t* s, int64_t n, int mode,
                 const Table& g, int32_t* slot2pool, int* err, cudaStream_t st);
// frame surface properties: per training point the mean of its voxel's point properties
void frame_point_props(const float* pts, const float* props, int64_t n, int nc, const DevParams& P, const Table& ft,
                       const unsigned long long* masks, const int32_t* slot2leaf, const int32_t* nocc,
                       const int64_t* inst_off, double* ysum, double* ycnt, cudaStream_t st);
void frame_prop_means(double* y, const double* ycnt, int64_t T, int nc, cudaStream_t st);

void fuse_alloc(int32_t* slot2pool, const Table& g, int* pool_count, int pool_cap, unsigned long long* known,
                int32_t* flags, int* err, const PropGrid& pg, cudaStream_t st);
void fuse_update(const uint64_t* vkey, const double* d, const double* v, const uint8_t* s, int64_t n, int mode,
                 const Table& g, const int32_t* slot2pool, unsigned long long* known, double* D, double* V,
                 int32_t* flags, const PropIn& pin, const PropGrid& pg, cudaStream_t st);
// properties of every known voxel (key order unspecified), and setting them for given keys
void grid_export_props(const Table& g, const int32_t* slot2pool, const unsigned long long* known, const PropGrid& pg,
                       int* count, uint64_t* okey, double* oC, double* oW, cudaStream_t st);
void grid_import_props(const uint64_t* vkey, const double* iC, const double* iW, int64_t n, const Table& g,
                       const int32_t* slot2pool, const unsigned long long* known, const PropGrid& pg, cudaStream_t st);
void grid_export(const Table& g, const int32_t* slot2pool, const unsigned long long* known, const double* D,
                 const double* V, const int32_t* flags, int* count, uint64_t* okey, double* oD, double* oV,
                 uint8_t* ofl, cudaStream_t st);
void grid_import(const uint64_t* vkey, const double* iD, const double* iV, const uint8_t* ifl, int64_t n, const Table& g,
                 int32_t* slot2pool, int* pool_count, int pool_cap, unsigned long long* known, double* D, double* V,
                 int32_t* flags, int* err, const PropGrid& pg, cudaStream_t st);
void grid_rehash(const Table& o, const int32_t* oslot2pool, const Table& nt, int32_t* nslot2pool, int* err,
                 cudaStream_t st);

}  // namespace vgp
