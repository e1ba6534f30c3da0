"""Paraxial optics helpers for the printers of Sec. 2.6 and Sec. 4 (test infrastructure).

These turn the paper's printed numbers into the geometry parameters the operators take
(pupil distance, image pixel pitch, cone half-angle) and back, so that the printed
values pin them.  Plain closed forms:
  thin lens (Sec. 2.6.1): image distance f(1+m), object distance f(1+1/m), m = image
      pixel / DMD pitch;
  divergence (Sec. 3.2): full cone angle 2*atan(D / (2 d)) for a stop of diameter D at
      distance d;
  etendue (Sec. 4): pixel area x solid angle with Omega = pi * theta^2, 2*theta the
      full divergence.
"""
import math


def magnification(image_pixel_mm: float, dmd_pitch_mm: float) -> float:
    return image_pixel_mm / dmd_pitch_mm


def thin_lens_image_distance(f_mm: float, m: float) -> float:
    return f_mm * (1.0 + m)


def thin_lens_object_distance(f_mm: float, m: float) -> float:
    return f_mm * (1.0 + 1.0 / m)


def full_divergence_deg(stop_diameter_mm: float, distance_mm: float) -> float:
    return math.degrees(2.0 * math.atan(stop_diameter_mm / (2.0 * distance_mm)))


def etendue_sr_mm2(pixel_mm: float, full_divergence_deg_: float) -> float:
    theta = math.radians(full_divergence_deg_) / 2.0
    return pixel_mm * pixel_mm * math.pi * theta * theta


def f_number_for_half_angle(half_angle_rad: float) -> float:
    """Working f-number N with tan(half-angle) = 1/(2N) (the operators' pupil model)."""
    return 1.0 / (2.0 * math.tan(half_angle_rad))
