// Degree-18 Taylor polynomial in five matrix products: the coefficients of
// B1 (I, A, A2, A3) and of B5, B4, B3, B2 (I, A, A2, A3, A6) in
//   A9 = B1 B5 + B4,   T = B2 + (B3 + A9) A9  =  sum_{k<=18} A^k / k!
// (the scheme of Bader, Blanes and Casas, Mathematics 7 (2019) 1174).
// Written by paper_2411_09982_gb300/taylor18_coefficients.py, which derives
// this member of the coefficient family and checks the 19 conditions; rounded
// to double they hold to 1.4e-16 relative.
#pragma once

namespace mg {
constexpr double kTaylor18[24] = {
    0.0010058693655587369,  // B1
    0.009404760087379685,  // B1
    0.0007523808069903748,  // B1
    8.359786744337498e-05,  // B1
    -1.759189225086304,  // B5
    -4.916424902717832,  // B5
    -2.3900877321888987,  // B5
    -0.024665646642923256,  // B5
    -0.00014949762421967295,  // B5
    -0.002230025728896113,  // B4
    0.08913048571509222,  // B4
    -0.017630637239739975,  // B4
    -0.012473559364650682,  // B4
    1.0206980602002909e-06,  // B4
    11.156502052331632,  // B3
    -1.680158138789062,  // B3
    -0.05717798464788655,  // B3
    0.0069821012248805206,  // B3
    -3.3497501708607054e-05,  // B3
    1.0446048830044943,  // B2
    0.23919036075055136,  // B2
    1.3624383975555403,  // B2
    0.49894895088677266,  // B2
    -0.0006410614046658537,  // B2
};
}  // namespace mg
