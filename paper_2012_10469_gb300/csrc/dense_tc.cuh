// Host interface of the tcgen05 dense product (dense_tc.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

struct SolveDev;

#define TC_NMAX 96          // 3 k padded to 16, k <= 32
#define TC_MAXG 24          // solves per launch (tensor maps travel as kernel parameters)

struct TcMaps {
    CUtensorMap a[TC_MAXG];   // over the objective's n x n bf16 data
    CUtensorMap b[TC_MAXG];   // over the split subspace block Wsp
};

#define TC_YS_SLOTS 8       // partial slots per solve: a tile is cut into at most this many segments

cudaError_t tc_init();
// resident CTAs of a launch over T chunks per SM (1 or 2); the ring shrinks to fit
int tc_ctas_per_sm(long long T, int sms);
bool tc_make_maps(const void* D, int n, const void* Wsp, int kpad, int npad, CUtensorMap* a, CUtensorMap* b);
// T = chunks of the launch (sum over its solves of row tiles x K chunks), G = CTAs
cudaError_t launch_dense_tc(const SolveDev* d_solves, int ns, long long T, int G, int npad_max, const TcMaps& maps,
                            cudaStream_t st);
