// Tiled single-pass kernel family (placeholder until the TMA kernel lands).
#include "lb_internal.h"

namespace lbhb {

struct TiledPlan {
    int dummy;
};

bool tiled_supported(const Geom&, int, int, int) { return false; }
int tiled_partials_nbx(const Geom& g, int tile_x) { return (g.nx + tile_x - 1) / tile_x; }
TiledPlan* tiled_create(const Geom&, int, int, void*, void*, int, int, const char** err_msg)
{
    if (err_msg) *err_msg = "tiled kernel not built";
    return nullptr;
}
void tiled_destroy(TiledPlan* p) { delete p; }
void tiled_tiles(const TiledPlan*, int* tx, int* ty) { *tx = *ty = 0; }
template <class T>
cudaError_t launch_tiled_step(TiledPlan*, int, const CellDev*, bool, double*, double*, unsigned*, cudaStream_t, int*)
{
    return cudaErrorNotSupported;
}
template cudaError_t launch_tiled_step<float>(TiledPlan*, int, const CellDev*, bool, double*, double*, unsigned*,
                                              cudaStream_t, int*);
template cudaError_t launch_tiled_step<double>(TiledPlan*, int, const CellDev*, bool, double*, double*, unsigned*,
                                               cudaStream_t, int*);
template cudaError_t launch_tiled_step<__half>(TiledPlan*, int, const CellDev*, bool, double*, double*, unsigned*,
                                               cudaStream_t, int*);
}  // namespace lbhb
