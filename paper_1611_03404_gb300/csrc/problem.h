// Host-side problem object shared by the library's translation units.
#pragma once

#include <string>
#include <vector>

#include "celeste_internal.cuh"

namespace celeste {

struct WsLayout {
  size_t images, patches, tiles, tile_pix, src_patch, nbr, u0, psf_coef, psf, pix, srcmom, ptab, partials, vpartials, flags, err, counters;
  size_t wl, wl_count, snc;
  size_t nt_f, nt_g, nt_H, nt_trial, nt_pred, nt_ftrial, nt_state, nt_count, nt_tcache, nt_lam, nt_list;
  size_t total;
};

int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
// Clears the bound problem's timeout word on st (at the start of every call that stages tiles).
cudaError_t clear_timeout(const ProblemDev& D, cudaStream_t st);
// Waits for st, then maps the problem's error words to a return code (CELESTE_OK when clear).
int device_errors(const ProblemDev& D, cudaStream_t st);

}  // namespace celeste

struct celeste_problem {
  int S = 0;
  int tile_pixels = 256;
  int hessian_mode = 0;
  long long wait_budget = 0;                          // celeste_problem_set_wait_budget (0: default)
  std::vector<celeste_image_desc> images;
  std::vector<double> u0;
  std::vector<int> radius;
  double priors[5];
  float nu[celeste::NMIX], tau[celeste::NMIX];
  // layout
  std::vector<celeste::PatchDev> patches;
  std::vector<celeste::TileDev> tiles;
  std::vector<long long> tile_pix;   // per tile: its patch's pixel offset + its start
  std::vector<int> src_patch, nbr;
  std::vector<celeste::ImageDev> imgdev;
  std::vector<double> psf_coef;
  long long n_pix = 0;
  celeste::WsLayout ws{};
  // binding
  char* base = nullptr;
  celeste::ProblemDev dev{};
  bool bound = false;
  bool background_ready = false;
  int background_mode = 0;                            // CELESTE_NBR_* of the last rendering
  // joint objective (built on first use): overlapping pairs, their overlap items and tiles
  bool joint_host_built = false, joint_built = false;   // host lists; uploaded to joint_dev
  std::vector<int> joint_pairs;                       // [n_pairs][2] sources s < t
  std::vector<int> joint_items_h, joint_tiles_h, joint_pair_items_h;   // flat int records
  int joint_n_items = 0, joint_n_tiles = 0;
  void* joint_dev = nullptr;                          // items, tiles, pair CSR, tile partials (caller memory)
  void* jn_dev = nullptr;                             // joint Newton state (caller memory, after the above)
  std::vector<int> jn_row_ptr_h, jn_row_ent_h;        // each source's coupling entries, uploaded at joint bind
  // profiling (celeste_profile_start/stop)
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_events;
  size_t prof_used = 0;
  std::vector<std::pair<int, int>> prof_full, prof_value;
  long long prof_launches = 0, prof_iters = 0;
  double prof_full_acc = 0.0, prof_value_acc = 0.0;   // ms of event pairs already read back
  double prof_tr_acc = 0.0;                           // ms of trust-region step launches
  long long prof_full_n = 0, prof_value_n = 0, prof_tr_n = 0;
  // Newton iterations as a CUDA graph (celeste_newton_batch), kept while its arguments repeat
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t newton_exec = nullptr;
  std::vector<unsigned char> newton_key;
  std::vector<cudaEvent_t> iter_events;               // 6 per captured iteration
  ~celeste_problem();
};

namespace celeste {
void build_layout(celeste_problem* p);
// Records an event on st when profiling; returns its index or -1.
int prof_mark(celeste_problem* p, cudaStream_t st);
inline void prof_count(celeste_problem* p, int launches) {
  if (p->prof_on) p->prof_launches += launches;
}
}
