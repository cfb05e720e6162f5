// kernels_f32.cu -- stage kernels instantiated with T = float.
#include "kernels.cuh"

namespace dg {

void upload_tables_f32(const Tab<double> td[2]) { upload_tables_tu(td); }

void launch_forcing_f32(const DevMesh &m, const Phys &ph, const Clock &clk, double tau, double t_fixed,
                        void *frc, const LaunchCfg &c) {
  launch_forcing_t<float>(m, ph, clk, tau, t_fixed, frc, c);
}
void launch_edge_f32(int p, const DevMesh &m, const StageArgs &s, const Phys &ph, const LaunchCfg &c) {
  launch_edge_t<float>(p, m, s, ph, c);
}
void launch_element_f32(int p, bool split, bool write_rhs, const DevMesh &m, const StageArgs &s,
                        const Phys &ph, const LaunchCfg &c) {
  launch_element_t<float>(p, split, write_rhs, m, s, ph, c);
}
void launch_limwd_f32(int p, bool do_lim, int do_wd, const DevMesh &m, double *u, const void *mean,
                      uint8_t *wd, const Phys &ph, int *err, const LaunchCfg &c, const uint8_t *cls) {
  launch_limwd_t<float>(p, do_lim, do_wd, m, u, mean, wd, ph, err, c, cls);
}

cudaError_t launch_ensemble_f32(int p, bool persistent, const EnsArgs &a, int block, int grid, cudaStream_t s) {
  return launch_ensemble_t<float>(p, persistent, a, block, grid, s);
}
int ensemble_blocks_per_sm_f32(int p, int block, bool ef) { return ensemble_blocks_per_sm_t<float>(p, block, ef); }

void launch_tile_f32(int p, bool wide, bool write_rhs, const DevMesh &m, const DevTiles &tl, const StageArgs &s,
                     const Phys &ph, const LaunchCfg &c) {
  launch_tile_t<float>(p, wide, write_rhs, m, tl, s, ph, c);
}
void prepare_tile_f32() { prepare_tile_t<float>(); }
void launch_front(int p, const DevMesh &m, const StageArgs &s, const Phys &ph, int write_rhs, cudaStream_t st) {
  launch_front_t(p, m, s, ph, write_rhs, st);
}
void launch_limwd_front(int p, bool do_lim, int do_wd, const DevMesh &m, double *u, const double *mean64,
                        const uint8_t *cls, uint8_t *wd, const Phys &ph, int *err, const int *flist,
                        const unsigned *fcnt, cudaStream_t st) {
  launch_limwd_front_t(p, do_lim, do_wd, m, u, mean64, cls, wd, ph, err, flist, fcnt, st);
}
void launch_copy_means_f32(int p, int ne, const double *u, void *mean, cudaStream_t s) {
  launch_copy_means_t<float>(p, ne, u, mean, s);
}

}  // namespace dg
