// tri_internal.h -- the unstructured constant-strain-triangle path of libcem
// (not part of the public ABI; cem_tri_mesh_create in include/cem.h is).
#pragma once

#include <string>

#include "cem.h"

namespace cem {

struct TriMesh;

// nullptr and a message in err on bad input or a CUDA failure
TriMesh *tri_create(const cem_tri_mesh_desc *desc, std::string &err);
void tri_destroy(TriMesh *t);
int tri_n_edges(const TriMesh *t);
cem_status tri_set_material(TriMesh *t, double E, double nu, double rho, int plane_strain,
                            const float *gc, double gc_uniform, double gamma, int gamma_mode,
                            std::string &err);
cem_status tri_set_bc(TriMesh *t, int kind, int n, const int *items, int comp_mask, int law,
                      double a0, double t0, double tau, std::string &err);
cem_status tri_set_fields(TriMesh *t, int which, const void *data, long n_bytes, int on_device,
                          std::string &err);
cem_status tri_step(TriMesh *t, int n, std::string &err);
cem_status tri_get_fields(TriMesh *t, int which, void *out, long n_bytes, int on_device,
                          std::string &err);
cem_status tri_eval_surface(TriMesh *t, int n, const int *edge, const int *elem, double *G,
                            int *choice, std::string &err);
void tri_counts(const TriMesh *t, cem_counts *out);

}  // namespace cem
