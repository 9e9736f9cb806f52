// Fused V(1,1) multigrid kernels: tile-shape queries, the automatic shape
// choice, the inverse diagonal, and the kernels' one-time setup.
#include "vfused.cuh"

namespace helm {

template <typename C>
void launch_make_dinv(const LevelView<double> &L, OpShift<double> s, C *dinv, cudaStream_t st) {
    const size_t N = (size_t)L.nx * L.ny * L.nz;
    const size_t b = (N + 255) / 256;
    const int nb = (int)(b < 4096 ? (b ? b : 1) : 4096);
    k_make_dinv<C><<<nb, 256, 0, st>>>(L, s, dinv);
    count_launch();
}
template void launch_make_dinv<double2>(const LevelView<double> &, OpShift<double>, double2 *, cudaStream_t);
template void launch_make_dinv<float2>(const LevelView<double> &, OpShift<double>, float2 *, cudaStream_t);

int num_tile_shapes(int dim) {
    return dim == 2 ? (int)n_down<2>() : dim == 3 ? (int)n_down<3>() : 0;
}

bool tile_shape(int dim, int kernel, int shape, int ext[3], int *threads, int *rb) {
    if (shape < 0 || shape >= num_tile_shapes(dim) || (kernel != 0 && kernel != 1)) return false;
    int rb_ = 1;
    if (dim == 2)
        shape_info<2>(kernel == 1, shape, ext, threads, &rb_, std::make_index_sequence<n_down<2>()>{});
    else
        shape_info<3>(kernel == 1, shape, ext, threads, &rb_, std::make_index_sequence<n_down<3>()>{});
    if (rb) *rb = rb_;
    return true;
}

int auto_tile_shape(int dim, int kernel, const int fine[3], int nb) {
    const int ns = num_tile_shapes(dim);
    const int cn[3] = {(fine[0] + 1) / 2, (fine[1] + 1) / 2, (fine[2] + 1) / 2};
    const int *ext_of = cn;                        // both kernels tile the coarse nodes
    long long best_blocks = -1;
    int best = 0;
    for (int sh = 0; sh < ns; ++sh) {
        int e[3], nt, rb;
        tile_shape(dim, kernel, sh, e, &nt, &rb);
        long long blocks = (long long)((nb + rb - 1) / rb) * ((ext_of[0] + e[0] - 1) / e[0]) *
                           ((ext_of[1] + e[1] - 1) / e[1]);
        if (dim == 3) blocks *= (ext_of[2] + e[2] - 1) / e[2];
        if (blocks >= 2 * (long long)device_sms()) return sh;
        if (blocks > best_blocks) {
            best_blocks = blocks;
            best = sh;
        }
    }
    return best;
}

void prepare_vfused() {
    // once per process, also when several threads (server workers) build
    // their grids at the same time
    static const int once = [] {
        vfused_attr_f64();
        vfused_attr_mixed();
        vfused_attr_c64();
        vfused_attr_ds();
        return 1;
    }();
    (void)once;
}

}  // namespace helm
