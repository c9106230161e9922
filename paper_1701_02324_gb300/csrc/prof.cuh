// prof.cuh -- launch accounting and optional per-phase timing.
//
// Every kernel launch of the library goes through KF_PHASE(phase, stream,
// launch): it bumps a process-wide launch counter and, while timing is on
// (kf_profile_enable), brackets the launch with CUDA events recorded on the
// launching stream.  kf_profile_read() synchronizes those events and returns
// per-phase totals.
#pragma once
#include <cuda_runtime.h>

enum kf_phase {
  KF_PH_TREE = 0,
  KF_PH_SAMPLE,
  KF_PH_EVAL_A,
  KF_PH_QR,
  KF_PH_LEAF_ASM,
  KF_PH_LEAF_CHOL,
  KF_PH_LEAF_PHAT,
  KF_PH_EVAL_V,
  KF_PH_ZOFF,
  KF_PH_ZLU,
  KF_PH_ZSOLVE_PC,
  KF_PH_TELESCOPE,
  KF_PH_S_LEAF,
  KF_PH_S_COLSUM,
  KF_PH_S_ZSOLVE,
  KF_PH_S_ROWUPD,
  KF_PH_MV_LEAF,
  KF_PH_MV_PUSH,
  KF_PH_MISC,
  KF_PH_QR_CLUSTER,
  KF_PH_QR_LEAF,
  KF_PH_MV_COLSUM,
  KF_PH_MV_ROWUPD,
  KF_PH_ZINV,
  KF_PH_HYBRID,
  KF_PH_NEAR,
  KF_PH_COUNT
};

void kf_prof_begin(int phase, cudaStream_t s);
void kf_prof_end(int phase, cudaStream_t s);

#define KF_PHASE(ph, stream, ...)   \
  do {                              \
    kf_prof_begin((ph), (stream));  \
    __VA_ARGS__;                    \
    kf_prof_end((ph), (stream));    \
  } while (0)
