// Per-kernel-class timing with CUDA events (off unless enabled) and a global
// count of kernel launches.  A scope records an event pair around the launches
// it encloses on the given stream and adds the class's algorithmic bytes.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace hedap {

enum ProfClass { PROF_NTT = 0, PROF_MODUP, PROF_KSK_INNER, PROF_MODDOWN, PROF_TENSOR, PROF_RESCALE,
                 PROF_AUTOMORPH, PROF_ELEMENTWISE, PROF_N_CLASSES };

void prof_count_launches(int n);
uint64_t prof_launches();
void prof_enable(bool on);
bool prof_enabled();
void prof_reset();
// sum of event-timed milliseconds, enclosed launches and algorithmic bytes of a class (synchronises)
void prof_read(int cls, uint64_t* scopes, double* ms, double* bytes);
// the same class's algorithmic multiply work in 32-bit multiply-pipe slots (see ProfScope::slots)
double prof_read_slots(int cls);
int prof_class_of(const char* name);

struct ProfScope {
  int cls;
  cudaStream_t st;
  double bytes;
  double slots = 0;  // algorithmic multiply work of the enclosed launches, in 32-bit multiply-pipe slots
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(int cls_, cudaStream_t st_, double bytes_);
  ~ProfScope();
};

}  // namespace hedap
