// Fused V(1,1) level kernels instantiated for the complex64 V-cycle on a
// complex64 basis (MIXED_C64), and that form's level-0 down kernel that forms
// v = w / ||w|| from the double-single w as it loads it.
#include "vfused.cuh"

namespace helm {

void vfused_attr_c64() {
    set_attr<float, float2>();
    set_attr_all_c64w<2>(std::make_index_sequence<n_down<2>()>{});
}

HELM_INST_V(float, float2)

bool launch_vdown_c64w(const LevelView<float> &F, const LevelView<float> &Cv, float wj, const float4 *w,
                       size_t sw, const float2 *sc, float2 *vout, size_t svout, float2 *u, size_t su, float2 *bc,
                       size_t sbc, int nb, const int *active, cudaStream_t st, int shape) {
    // 2D only: the 3D tiles load a halo of about 2.25x their own nodes, and
    // loading w (16 B) there in place of v (8 B) cost more than the separate
    // scaling kernel it saves (126 against 91 + 31 ms in the 4-source
    // 257 x 257 x 193 solve)
    if (F.dim != 2) return false;
    prof_begin(st);
    const bool ok = down_c64w_sel<2>(shape, std::make_index_sequence<n_down<2>()>{}, F, Cv, wj, w, sw, sc, vout,
                                     svout, u, su, bc, sbc, nb, active, st);
    if (prof_on()) {
        // per right-hand side: w in (16 B), v and u out (8 B each), the coarse
        // right-hand side out; D^-1 once per launch
        const double n1 = (double)F.nx * F.ny * F.nz;
        const double nf = n1 * nb, nc = (double)Cv.nx * Cv.ny * Cv.nz * nb;
        prof_end("vdown_l0_f32", st, nf * 32.0 + n1 * 8.0 + nc * 8.0, 0.0);
    }
    return ok;
}

}  // namespace helm
