// Library-wide entry points: status strings, version, and the conversion of
// the host robot description into the kernels' parameter block.
#include <cuda_runtime.h>

#include <cmath>

#include "fn_arm.cuh"
#include "fn_internal.h"

namespace fn {

bool make_armk(const fn_arm_t* a, ArmK* o) {
  if (!a || !o || a->dof != FN_DOF) return false;
  for (int j = 0; j < 7; ++j) {
    if (!(a->tau_max[j] > 0.f) || !(a->qd_max[j] >= 0.f) || !(a->q_hi[j] >= a->q_lo[j]) ||
        !(a->qd_taper_a[j] >= 0.f))
      return false;
    const double al = a->dh_alpha[j];
    const double ca = std::cos(al), sa = std::sin(al);
    o->ca[j] = (float)ca;
    o->sa[j] = (float)sa;
    o->px[j] = a->dh_a[j];
    o->py[j] = (float)(-sa * (double)a->dh_d[j]);
    o->pz[j] = (float)(ca * (double)a->dh_d[j]);
    o->th0[j] = a->dh_theta0[j];
    o->m[j] = a->mass[j];
    o->cx[j] = a->com[j][0];
    o->cy[j] = a->com[j][1];
    o->cz[j] = a->com[j][2];
    o->Ix[j] = a->inertia[j][0];
    o->Iy[j] = a->inertia[j][1];
    o->Iz[j] = a->inertia[j][2];
    o->arma[j] = a->armature[j];
    o->f1[j] = a->fric[j][0];
    o->f2[j] = a->fric[j][1];
    o->f3[j] = a->fric[j][2];
    // tau_f(0) = 0: the constant term psi1 * sigmoid(psi2 psi3), in double
    o->foff[j] = (float)((double)a->fric[j][0] /
                         (1.0 + std::exp(-(double)a->fric[j][1] * (double)a->fric[j][2])));
    o->inv_tau[j] = (float)(1.0 / (double)a->tau_max[j]);
    o->q_lo[j] = a->q_lo[j];
    o->q_hi[j] = a->q_hi[j];
    o->qd_max[j] = a->qd_max[j];
    o->taper2a[j] = 2.0f * a->qd_taper_a[j];
    o->lrad[j] = a->link_radius[j];
  }
  if (!(a->w_max > 0.f)) return false;
  o->inv_w = (float)(1.0 / (double)a->w_max);
  o->g0x = -a->gravity[0];
  o->g0y = -a->gravity[1];
  o->g0z = -a->gravity[2];
  o->flange_d = a->flange_d;
  for (int k = 0; k < 3; ++k) {
    o->bb[k] = a->blade_base[k];
    o->bax[k] = a->blade_axis[k];
    o->bnm[k] = a->blade_normal[k];
  }
  o->blen = a->blade_len;
  return true;
}

}  // namespace fn

extern "C" const char* fn_status_str(int s) {
  switch (s) {
    case FN_OK: return "FN_OK";
    case FN_EINVAL: return "FN_EINVAL: invalid argument";
    case FN_ECUDA: return "FN_ECUDA: CUDA call or launch failed";
    case FN_ENOMEM: return "FN_ENOMEM: allocation failed";
    case FN_ETIMEOUT: return "FN_ETIMEOUT: bounded device wait gave up";
    case FN_EDEADLINE: return "FN_EDEADLINE: host deadline expired";
    default: return "unknown status";
  }
}

extern "C" const char* fn_version(void) { return "fruitninja-gb300 0.1 (sm_103a)"; }
