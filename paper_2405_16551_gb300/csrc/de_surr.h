// de_surr.h -- surrogate-assisted generations (de_surr.cu): k candidate
// trials per target, screened by the surrogate network, one true evaluation
// per target, an archive of (trial, f) rows for online training.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include <string>
#include <vector>

#include "de.h"
#include "de_internal.cuh"
#include "de_mlp.h"

namespace de {

// Network object of de_mlp.cu, used by the surrogate loop.
de_status mlp_create(uint64_t seed, cudaStream_t stream, ::de_mlp** out);
void mlp_destroy(::de_mlp* m);
de_status mlp_reset(::de_mlp* m);
const MlpDev& mlp_dev(const ::de_mlp* m);
de_status mlp_train_rows(::de_mlp* m, const double* x, int64_t ld, const float* t, int n, int base, int cap, int steps,
                         float lr);

// Settings (choices of this implementation; the paper has no surrogate):
//   warm-up of `warmup` plain generations, then retraining every `retrain`
//   generations on the most recent `window` archive rows with `steps` Adam
//   steps (lr 1e-3, minibatch 256) on standardised log(f); screening with k
//   candidates only while the Spearman correlation between the network's
//   prediction and the true f of the last generation's evaluated trials is at
//   least rho_min (otherwise one candidate, i.e. plain DE).
struct Surrogate {
  int k = 8;
  int steps = 25;  // Adam steps per retraining (the default of surrogate_steps)
  float lr = 1e-3f;
  int warmup = 5, retrain = 10, window = 20000, cap = 200000;
  double rho_min = 0.3;
  ::de_mlp* mlp = nullptr;
  void* arena = nullptr;
  double* C = nullptr;        // np * k candidate rows (stride dp)
  double* T = nullptr;        // np evaluated trials (stride dp)
  double* ftrial = nullptr;   // np true fitness values of T
  float* yhat = nullptr;      // np * k predictions
  float* yhat_sel = nullptr;  // np predictions of the evaluated trials
  int32_t* cand_sel = nullptr;
  double* arch_x = nullptr;   // cap archive rows (stride dp)
  double* arch_f = nullptr;   // their true fitness
  float* arch_t = nullptr;    // training targets of the current window
  std::vector<double> h_f, h_win;
  std::vector<float> h_y;
  long long head = 0, count = 0, gens = 0, since_train = 0, trainings = 0, screened = 0;
  int k_eff = 1;
  bool trained = false;
  double last_rho = NAN;
};

de_status surr_create(Surrogate*& S, int k, int steps, uint64_t seed, const RunDesc& R, cudaStream_t s,
                      std::string& err);
void surr_destroy(Surrogate* S);
de_status surr_reset(Surrogate& S, cudaStream_t s, std::string& err);
// One generation of run 0 (synchronises the stream).
de_status surr_generation(Surrogate& S, const RunDesc* d_run, const RunDesc& R, cudaStream_t s, std::string& err);

}  // namespace de
