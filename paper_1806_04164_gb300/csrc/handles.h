// Definitions of the opaque handles of include/pie.h.
#pragma once
#include "problem.h"

struct pie_mesh {
  pie::Mesh m;
};
struct pie_problem {
  pie::Problem p;
};
