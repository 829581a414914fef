// Learned step-cost model (costmodel.cu) and the step features it reads.
#pragma once
#include <vector>

#include "tn.h"

namespace tn {

constexpr int kCostFeatures = 16;
// feature 14 = log2(roofline time in ms) / kRoofFeatureScale; the model
// predicts log2(step time / roofline time)
constexpr double kRoofFeatureScale = 16.0;

// number of MLP parameters
int cost_params();

// model outputs (log2 of time over roofline time) for a host feature matrix (rows of kCostFeatures);
// synchronous, on the legacy stream
int cost_predict_host(tn_costmodel_t cm, const std::vector<float> &X, std::vector<float> &Y);

}  // namespace tn
