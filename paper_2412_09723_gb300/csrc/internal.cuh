// internal.cuh -- kernel-side views of the ABI structs and launcher
// declarations shared between the translation units of the library.
#pragma once

#include "common.cuh"

namespace splat {

struct CamK {
  int width, height, tiles_x, tiles_y;
  float fx, fy, cx, cy, znear;
  float maxd2;  // squared distance limit, 0 = none
};

struct GaussiansK {
  const float* mean;
  const float* log_scale;
  const float* quat;
  const float* opacity_logit;
  const float* rgb;
  int64_t n;
};

struct ProjectedK {
  float* xyzo;
  float* conic;
  int32_t* radius;
  int32_t* rect;
  int32_t* tiles_touched;
};

struct GradK {
  float* mean;
  float* log_scale;
  float* quat;
  float* opacity_logit;
  float* rgb;
};

inline CamK make_camk(const splat_camera& c) {
  CamK k;
  k.width = c.width;
  k.height = c.height;
  k.tiles_x = (c.width + kTile - 1) / kTile;
  k.tiles_y = (c.height + kTile - 1) / kTile;
  k.fx = c.fx; k.fy = c.fy; k.cx = c.cx; k.cy = c.cy; k.znear = c.z_near;
  k.maxd2 = c.max_dist > 0.f ? c.max_dist * c.max_dist : 0.f;
  return k;
}

int launch_project_fwd(const GaussiansK& g, const CamK& cam, const float* w2c, const ProjectedK& out,
                       cudaStream_t s);
// g2: screen-space gradients, rows of `stride` floats (du, dv, d conic a, b, c,
// d opacity, d rgb[3], d depth, padding); d2d_out (optional): copy [n,10].
// radius: the forward projection's radii (0 = culled: no gradient, skipped).
int launch_project_bwd(const GaussiansK& g, const CamK& cam, const float* w2c, const float* conic,
                       const int32_t* radius, const float* g2, int stride, const GradK& out, float* d_pose,
                       float* d2d_out, cudaStream_t s);

// L1 terms: grgb = sc sign(rgb - trgb), gdepth = sd sign(depth - tdepth) (overwritten),
// loss += sc sum|rgb - trgb| + sd sum|depth - tdepth|.
int launch_loss_l1(const float* rgb, const float* depth, const float* trgb, const float* tdepth, int64_t npix,
                   float sc, float sd, float* grgb, float* gdepth, float* loss, cudaStream_t s);

}  // namespace splat
