// Library-internal interface between the solver core (api.cu) and the request
// server (serve.cu): resumable solves on a handle and device-memory accounting.
#pragma once
#include <cuda_runtime.h>

#include "helm.h"

namespace helm {
struct Task;   // one FGMRES solve as a resumable state machine on the handle's stream
int task_create(helm_t h, const double2* F, double2* x, Task** out);
// Advances the solve; returns true once it has finished (res, rc filled).
bool task_step(Task* k, bool blocking, helm_result* res, int* rc);
void task_destroy(Task* k);
size_t handle_bytes(helm_t h);
size_t estimate_bytes(int dim, int order, int n, int precision, int restart);
}  // namespace helm
