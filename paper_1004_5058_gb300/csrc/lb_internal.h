// Internal launch interface between the C ABI (lb_capi.cu) and the kernels.
#pragma once

#include "lb_common.cuh"

namespace lbhb {

// generic family (lb_generic.cu)
template <class T>
cudaError_t launch_generic_step(const T* fin, T* fout, const Geom& g, int bc, const CellDev* cells, void* aux,
                                bool sample, double* prof_part, double* wall_part, unsigned* err,
                                cudaStream_t st, int* n_launches);
int generic_partials_nbx(const Geom& g);

// tiled family (lb_tiled.cu)
struct TiledPlan;  // opaque per-handle state of the tiled kernel
bool tiled_supported(const Geom& g, int elem_bytes, int tile_x, int tile_y);
int tiled_partials_nbx(const Geom& g, int tile_x);
// Creates the plan (tensor maps for both ping-pong buffers).  Returns nullptr
// and sets *err_msg if the shape/tile is not supported or encoding failed.
// g: the whole population buffer; rm: the rows a step updates (a whole cell, or
// the own rows of a slab between its ghost rows).
TiledPlan* tiled_create(const Geom& g, const RowMap& rm, int prec, int elem_bytes, int bc, void* f0, void* f1,
                        int tile_x, int tile_y, const char** err_msg);
void tiled_destroy(TiledPlan* p);
template <class T>
cudaError_t launch_tiled_step(TiledPlan* p, int src_buf, const CellDev* cells, bool sample, double* prof_part,
                              double* wall_part, unsigned* err, cudaStream_t st, int* n_launches);
void tiled_tiles(const TiledPlan* p, int* tx, int* ty);
// Persistent CTAs of plain and sampled launches of the family that runs, threads
// per CTA and dynamic shared memory per CTA (outputs nullable).
void tiled_launch_shape(const TiledPlan* p, int* grid_plain, int* grid_sampled, int* threads, int* smem);
// Failure injection (tests): the next launch's CTA 0 leaves the copy of its row
// `row` (counted over its work items) unissued, so the waits for it time out.
void tiled_inject_skip(TiledPlan* p, uint32_t row);
// The cells' collision: BGK with one relaxation time for every cell (the
// full-width kernels serve only that case), BGK with a time per species in some
// cell (the general kernels), or multiple relaxation times in some cell (the
// MRT kernels, which then run every cell of the batch).
enum { TILED_BGK_ONE_TIME = 0, TILED_BGK = 1, TILED_MRT = 2 };
void tiled_set_collision(TiledPlan* p, int collision);

// auxiliary kernels (lb_aux.cu)
template <class T>
cudaError_t launch_equilibrium(const double* src, T* f, const Geom& g, const CellDev* cells, cudaStream_t st);
template <class T>
cudaError_t launch_export(const T* f, double* dst, const Geom& g, const CellDev* cells, cudaStream_t st);
template <class T>
cudaError_t launch_import(const double* src, T* f, const Geom& g, const CellDev* cells, cudaStream_t st);
template <class T>
cudaError_t launch_fields(const T* f, double* dst, const Geom& g, const CellDev* cells, unsigned* err,
                          cudaStream_t st);
int state_sums_blocks(const Geom& g);
template <class T>
cudaError_t launch_state_sums(const T* f, const Geom& g, const CellDev* cells, double* part, double* out,
                              unsigned* err, cudaStream_t st);
cudaError_t launch_accumulate(const double* prof_part, const double* wall_part, int nbx, int ny, int bc,
                              int n_cells, double* acc_prof, double* acc_wall, cudaStream_t st);

// Slab exchange (lb_aux.cu): n_planes of the 18 planes, rows [row0, row0 + nrows)
// of the buffer g of every cell, to (pack) or from a dense message.
struct SlabMsg {
    int n_planes, row0, nrows;
    int planes[18];
};
template <class T>
cudaError_t launch_slab_msg(T* f, T* msg, const Geom& g, const SlabMsg& m, bool pack, cudaStream_t st);

// A caller's device buffer (lb_noalloc.cu): device or managed memory of device
// `dev` whose allocation holds `bytes` bytes from p on.  false and a reason in
// why otherwise.
bool device_buffer_ok(const void* p, size_t bytes, int dev, const char* name, char* why, size_t why_len);

// Message returned by lb_last_error(NULL) (lb_capi.cu).
void set_handleless_error(const char* msg);

}  // namespace lbhb
