// pgvimp_launch.h -- launch groups of the hot-path kernels (internal).
#pragma once
#include "pgvimp_plan.h"
#include "pgvimp_device.cuh"

namespace pgv {
template <int n, typename QT, typename R> cudaError_t launch_iter(const Launch& L, int iters);
template <int n, typename R> cudaError_t launch_aux(const Launch& L, int phase, int arg_i, int qt32);
template <int n> cudaError_t launch_rows(const Launch& L, int phase, double arg_d, int mixed);
template <int n, typename QT, typename R> cudaError_t launch_iter_cta(const Launch& L, int iters, int tpb);
template <typename QT, typename R> cudaError_t launch_iter_lane(const Launch& L, int iters);   // n = 4
extern template cudaError_t launch_iter_lane<float, df64>(const Launch&, int);
extern template cudaError_t launch_iter_lane<float, double>(const Launch&, int);
extern template cudaError_t launch_iter_lane<double, double>(const Launch&, int);
template <int n, typename R> cudaError_t launch_aux_cta(const Launch& L, int phase, int arg_i, int qt32, int tpb);
extern template cudaError_t launch_iter<4, float, double>(const Launch&, int);
extern template cudaError_t launch_iter<4, double, double>(const Launch&, int);
extern template cudaError_t launch_iter<4, float, df64>(const Launch&, int);
extern template cudaError_t launch_aux<4, double>(const Launch&, int, int, int);
extern template cudaError_t launch_aux<4, df64>(const Launch&, int, int, int);
extern template cudaError_t launch_rows<4>(const Launch&, int, double, int);
extern template cudaError_t launch_iter<6, float, double>(const Launch&, int);
extern template cudaError_t launch_iter<6, double, double>(const Launch&, int);
extern template cudaError_t launch_iter<6, float, df64>(const Launch&, int);
extern template cudaError_t launch_aux<6, double>(const Launch&, int, int, int);
extern template cudaError_t launch_aux<6, df64>(const Launch&, int, int, int);
extern template cudaError_t launch_rows<6>(const Launch&, int, double, int);
extern template cudaError_t launch_iter<14, float, double>(const Launch&, int);
extern template cudaError_t launch_iter<14, double, double>(const Launch&, int);
extern template cudaError_t launch_iter<14, float, df64>(const Launch&, int);
extern template cudaError_t launch_aux<14, double>(const Launch&, int, int, int);
extern template cudaError_t launch_aux<14, df64>(const Launch&, int, int, int);
extern template cudaError_t launch_rows<14>(const Launch&, int, double, int);
extern template cudaError_t launch_iter_cta<4, float, double>(const Launch&, int, int);
extern template cudaError_t launch_iter_cta<4, double, double>(const Launch&, int, int);
extern template cudaError_t launch_aux_cta<4, double>(const Launch&, int, int, int, int);
extern template cudaError_t launch_iter_cta<4, float, df64>(const Launch&, int, int);
extern template cudaError_t launch_aux_cta<4, df64>(const Launch&, int, int, int, int);
extern template cudaError_t launch_iter_cta<6, float, double>(const Launch&, int, int);
extern template cudaError_t launch_iter_cta<6, double, double>(const Launch&, int, int);
extern template cudaError_t launch_aux_cta<6, double>(const Launch&, int, int, int, int);
extern template cudaError_t launch_iter_cta<6, float, df64>(const Launch&, int, int);
extern template cudaError_t launch_aux_cta<6, df64>(const Launch&, int, int, int, int);
extern template cudaError_t launch_iter_cta<14, float, double>(const Launch&, int, int);
extern template cudaError_t launch_iter_cta<14, double, double>(const Launch&, int, int);
extern template cudaError_t launch_aux_cta<14, double>(const Launch&, int, int, int, int);
extern template cudaError_t launch_iter_cta<14, float, df64>(const Launch&, int, int);
extern template cudaError_t launch_aux_cta<14, df64>(const Launch&, int, int, int, int);
}  // namespace pgv
