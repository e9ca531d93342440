// Launchers of the midpoint predict-evaluate-correct integrator (pec.cu).
#pragma once

#include <cuda_runtime.h>

#include "sph_launch.h"

namespace sph {

// Predictor on the current order, in place: saves (x, u, rho) of every particle into
// `save` ((2 dim + 1) arrays of n doubles) and the step size *idt into *dt_step, then
// advances to the half step. continuity: the density is integrated (else summation).
void launch_pec_predict(const ParticleSet& S, double* save, int n, int dim, const Grid& G,
                        const double* idt, double* dt_step, int continuity, const Control* ctl,
                        int sms, cudaStream_t st);

// Corrector on the order of the midpoint build: particle k finds its saved state at
// perm[k] (its position before that build) and takes the full step with the rates of the
// midpoint evaluation.
void launch_pec_correct(const ParticleSet& S, const double* save, const uint32_t* perm, int n,
                        int dim, const Grid& G, const double* dt_step, int continuity,
                        const Control* ctl, int sms, cudaStream_t st);

// After the end-of-step evaluation: advances t and the step count by the step just taken
// and appends the diagnostics record to the history.
void launch_pec_record(Control* ctl, double* history, const double* dt_step, cudaStream_t st);

// Batch forms: each particle takes the grid and step size of its instance (found from its
// cell key in skeys, the keys of the order the kernel works on); dt_step holds one step
// size per instance. The record advances every instance's t and step count.
void launch_pec_predict_batch(const ParticleSet& S, double* save, int n, int dim, int precision,
                              const void* tab, const uint32_t* cell_bounds, int ninst,
                              const uint32_t* skeys, const double* idt, double* dt_step,
                              int continuity, const Control* ctl, int sms, cudaStream_t st);
void launch_pec_correct_batch(const ParticleSet& S, const double* save, const uint32_t* perm, int n,
                              int dim, int precision, const void* tab, const uint32_t* cell_bounds,
                              int ninst, const uint32_t* skeys, const double* dt_step,
                              int continuity, const Control* ctl, int sms, cudaStream_t st);
void launch_pec_record_batch(double* it, double* irec, const double* dt_step, int ninst,
                             const Control* ctl, cudaStream_t st);

}  // namespace sph
