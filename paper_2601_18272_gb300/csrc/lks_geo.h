// Problem validation and the problem constants (Geo) of the library, shared by lks_create and the
// allocation-free step so that both derive the same geometry from one lks_problem.
#pragma once

#include "../../include/lks.h"
#include "lks_device.cuh"

namespace lks {

// LKS_OK if the problem is one lks_create accepts, else its status (LKS_ERR_ARG,
// LKS_ERR_UNSTABLE, LKS_ERR_UNSUPPORTED).
int validate_problem(const lks_problem* P);

// The problem constants of a validated problem, with the body box sized as lks_create sizes it:
// the rotated (circumscribed) box when it fits every periodic extent, else the axis-aligned box
// for a body without the rotational DOF. *rot_ok tells whether the rotated box fits (a body may
// start rotated only then). LKS_ERR_UNSUPPORTED if no box fits.
int make_geometry(const lks_problem* P, Geo* g, bool* rot_ok);

// Body box of g for the design domain of design_radius: circumscribed in the rotation plane (every
// axis with free rotation) if rotated, else axis-aligned.
void setup_box(Geo* g, double design_radius, bool rotated);

// True if the body box fits every periodic extent of the grid.
bool box_fits(const Geo& g);

// Tiles of box cells of the body kernels (16 x 16 cells in 2D, 16 x 8 per plane in 3D).
long long box_tiles(const Geo& g);

}  // namespace lks
