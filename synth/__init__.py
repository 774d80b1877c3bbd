"""Seeded synthetic input generators shared by the oracle, the tests and the benchmark."""
from .voronoi import (ImageSpec, make_image, make_image_f32, voronoi_labels, batch_specs,
                      PARITY_64_RGB, THROUGHPUT_1024_RGB, GRADIENT_2048_RGB)
from .params import init_net_params

__all__ = ["ImageSpec", "make_image", "make_image_f32", "voronoi_labels", "batch_specs",
           "PARITY_64_RGB", "THROUGHPUT_1024_RGB", "GRADIENT_2048_RGB", "init_net_params"]
